// Internal interface of the proposal-network training kernels.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace su {
namespace train {

// Device buffers of one training step on up to cap_rows rows (R multiple of 32).
struct Workspace {
    void *base = nullptr;
    int cap_rows = 0;
    __nv_bfloat16 *X = nullptr, *XT = nullptr;          // inputs [R][32], [32][R]
    float *u = nullptr, *rw = nullptr;                   // targets, row weights
    float *pre[3] = {nullptr, nullptr, nullptr};        // pre-activations [R][128]
    __nv_bfloat16 *H[3] = {nullptr, nullptr, nullptr};  // activations [R][128]
    __nv_bfloat16 *HT[3] = {nullptr, nullptr, nullptr}; // transposed [128][R]
    float *Y = nullptr;                                  // outputs [R][2] (no bias)
    __nv_bfloat16 *dYp = nullptr, *dYT = nullptr;        // dL/dY [R][32], [2][R]
    __nv_bfloat16 *dP = nullptr, *dPT = nullptr;         // dL/dpre [R][128], [128][R]
    __nv_bfloat16 *dP2 = nullptr, *dPT2 = nullptr;       // the same, the other layer of a pair
    __nv_bfloat16 *W1p = nullptr, *W2 = nullptr, *W3 = nullptr, *W4 = nullptr;
    __nv_bfloat16 *W2T = nullptr, *W3T = nullptr, *W4T = nullptr;
    float *dW1 = nullptr, *dW2 = nullptr, *dW3 = nullptr, *dW4 = nullptr, *db = nullptr;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;   // flat, kParams each
    double *loss = nullptr;
    int *status = nullptr;                               // set when a tensor-core wait gave up
    size_t grad_bytes = 0, gbytes = 0;

    ~Workspace();
    void release();
    cudaError_t reserve(int R);
};

// loss and flat gradient of the rows already in ws (X, XT, u, rw), at ws.theta
cudaError_t loss_grad(Workspace &ws, int R, double inv_norm, bool use_rw, cudaStream_t st);
// one Adam step (t >= 1) on ws.theta with ws.grad
cudaError_t adam_step(Workspace &ws, int t, float lr, cudaStream_t st);
// minibatch rows from stored paths ([n][np1] floats) of the listed path ids
cudaError_t build_rows(Workspace &ws, const float *paths, int np1, const int *ids, int nb, float a, float b,
                       float T, int S, const float *sig, cudaStream_t st);
// rows from given features (n x 6 floats), targets and weights; rows n..R-1 zero
cudaError_t rows_from_features(Workspace &ws, const float *X, const float *u, const float *rw, int n, int R,
                               cudaStream_t st);
cudaError_t fill(float *p, float v, int n, cudaStream_t st);
// minibatch path ids of step *step (device counter): nb draws in proportion to
// the weights whose running sums are cdf[0..n) (total = cdf[n-1]), Philox under
// the key seed
cudaError_t sample_ids(const double *cdf, int64_t n, double total, uint64_t seed, const int *step, int nb,
                       int *ids, cudaStream_t st);
// Adam step with t = *step + 1 taken from the device
cudaError_t adam_step_dev(Workspace &ws, const int *step, float lr, cudaStream_t st);
// losses[*step] = *loss, then ++*step
cudaError_t step_tail(int *step, const double *loss, double *losses, cudaStream_t st);

}  // namespace train
}  // namespace su
