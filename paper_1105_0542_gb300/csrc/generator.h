// Host-side generator of the level-p effective potential (internal header).
//
// The coefficients c_{m,k} of Eq. ansatz follow from Eq. 1Drec with the
// diagonal of Eq. diagonal, evaluated in the order of Fig. 1; they are kept as
// polynomials in one ring variable with double-double coefficients and then
// collapsed, for one eps, into the table the sampler evaluates per slice.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace su {

// Ring of the collapsed polynomial in x.
enum Ring : int {
    RING_EVEN = 0,   // z = x^2            (even polynomial potentials)
    RING_X = 1,      // z = x              (general polynomial potentials)
    RING_TANH2 = 2,  // z = tanh^2(alpha x)  (modified Poeschl-Teller)
};

struct Shape {
    int ring = RING_EVEN;
    int ncol = 0;                 // J + 1 columns (powers xb^(2j))
    std::vector<int> len;         // entries of column j (D_j + 1)
    int M = 0;                    // total entries
    double alpha = 0;             // for RING_TANH2
};

struct Effective {
    int p = 0;
    Shape shape;
    // c[m][k] as polynomial in the ring variable (x for RING_EVEN/RING_X,
    // s = tanh^2(alpha x) for RING_TANH2), stored as (hi, lo) pairs
    std::vector<std::vector<std::vector<double>>> hi, lo;
};

// Validates the model and builds c_{m,k}, m < p.  Returns SU_OK or an error
// code and message.
int build_effective(int model, const double *params, int n_params, int p, Effective &E,
                    std::string &err);

// P_{ij}(eps) = sum_{m} c_{m,j}[ring index i] eps^(m-j): W_p in the form
// sum_j xb^(2j) sum_i P_ij z^i (see speedup.h).  Fills P (shape.M entries).
void collapse(const Effective &E, double eps, std::vector<double> &P);

// The sampler's table for one level: entry (i, j) = -eps P_ij scaled to the
// kernel's variables us = q_k + q_{k+1} and vs = q_{k+1} - q_k, so that the
// per-slice contribution -eps W_p is sum_j (vs^2)^j sum_i T_ij Z^i with
// Z = us^2 (RING_EVEN), us (RING_X) or tanh^2(alpha us / 2) (RING_TANH2).
// Also returns the largest ratio sum|terms| / |sum| met while collapsing (a
// cancellation measure of the double-double sums).
double kernel_table(const Effective &E, double eps, std::vector<double> &T);

// W_p(x, xb; eps) evaluated on the host from the double-double collapse.
double wp_host(const Effective &E, double x, double xb, double eps);

// W_p(x, xb; eps) from a collapse P already made for that eps (double).
double wp_collapsed(const Shape &S, const std::vector<double> &P, double x, double xb);

}  // namespace su
