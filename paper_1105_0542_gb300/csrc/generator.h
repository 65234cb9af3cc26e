// Host-side generator of the level-p effective potential (internal header).
//
// The coefficients c_{m,k} of Eq. ansatz follow from Eq. 1Drec with the
// diagonal of Eq. diagonal, evaluated in the order of Fig. 1; they are kept as
// polynomials in one ring variable with double-double coefficients and then
// collapsed, for one eps, into the table the sampler evaluates per slice.
#pragma once

#include <cstdint>
#include <map>
#include <string>
#include <vector>

namespace su {

// Ring of the collapsed polynomial in x.
enum Ring : int {
    RING_EVEN = 0,   // z = x^2            (even polynomial potentials)
    RING_X = 1,      // z = x              (general polynomial potentials)
    RING_TANH2 = 2,  // z = tanh^2(alpha x)  (modified Poeschl-Teller)
    RING_GENERAL = 3,  // general potential: W_p in the derivative symbols V^(j)(x)
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

// W_p(x, xb; eps) evaluated on the host from the double-double collapse;
// the _points form collapses once for n points (w[i] at x[i], xb[i]).
double wp_host(const Effective &E, double x, double xb, double eps);
void wp_host_points(const Effective &E, double eps, const double *x, const double *xb, int64_t n, double *w);

// W_p(x, xb; eps) from a collapse P already made for that eps (double).
double wp_collapsed(const Shape &S, const std::vector<double> &P, double x, double xb);

// ---- general potentials: W_p as a polynomial in the derivative symbols
// V_j = V^(j)(x), j = 0..2p-2 (the same recursion with d/dx V_j = V_{j+1}).
// The distinct monomials of W_p form a trie over their non-decreasing symbol
// sequences; its nodes in depth-first order give an evaluation program in
// which every monomial is its parent (one level up) times one symbol.
constexpr int kGenMaxP = 18;   // the paper's compiled W_p reaches p = 18 (Sec. 3.1)

struct GeneralEffective {
    int p = 0;
    int J = 0;                        // highest symbol in W_p: 2p - 2
    int K = 0;                        // powers xb^(2k), k = 0..K-1
    std::vector<int> depth, sym;      // DFS nodes; node 0 is the constant monomial
    std::vector<int> first, count;    // node -> its entries [first, first + count)
    std::vector<int> entry_k;         // entry -> k
    // entry -> coefficient of eps^(m-k) for m = k..p-1 (hi, lo)
    std::vector<std::vector<double>> entry_hi, entry_lo;
};

int build_general(int p, GeneralEffective &G, std::string &err);

// The level table of the general program for one eps: entry e of power k
// gets -eps * sum_m c_m eps^(m-k) / 4^k (xb^(2k) = vs^(2k) / 4^k).
void general_table(const GeneralEffective &G, double eps, std::vector<double> &T);

// The potential of the general mode (SU_GENERAL): a polynomial of degree <= 8,
// up to four Gaussians A e^{-beta (x - c)^2}, four sech^2 terms
// B sech^2(alpha (x - d)) and, optionally, four exponentials
// E e^{-kappa (x - x0)}; parameters (a_0..a_8, (A, beta, c) x 4,
// (B, alpha, d) x 4 [, (E, kappa, x0) x 4]), terms with a zero amplitude absent.
constexpr int kGenParams = 9 + 3 * 4 + 3 * 4;
constexpr int kGenParamsExp = kGenParams + 3 * 4;
struct GeneralPotential {
    double a[9] = {0};
    int ng = 0, ns = 0, ne = 0;
    double gauss[4][3] = {{0}};   // A, beta, c
    double sech[4][3] = {{0}};    // B, alpha, d
    double expo[4][3] = {{0}};    // E, kappa, x0
};
int general_potential(const double *params, int n_params, GeneralPotential &V, std::string &err);

// V^(j)(x), j = 0..J, on the host (double).
void general_derivatives(const GeneralPotential &V, double x, int J, double *out);

// W_p(x, xb; eps) of the general potential on the host (level 0 and tests).
double general_wp_host(const GeneralEffective &G, const GeneralPotential &V, double x, double xb, double eps);
void general_wp_points(const GeneralEffective &G, const GeneralPotential &V, double eps, const double *x,
                       const double *xb, int64_t n, double *w);

// ---- systems of d = D x M coordinates (Sec. 2.2): the level-p effective
// potential W(x, xb; eps) of a polynomial potential V(x_1..x_d) by the
// contracted recursion (Eq. MBrec, diagonal Eq. DIA, Fig. 1 order) over
// polynomials in the 2d variables z = (x_1..x_d, xb_1..xb_d), in
// double-double.  For evaluation the distinct monomials are grouped by their
// part without one variable z_H (the one that makes the program shortest):
// a group is z_H^j0 times a polynomial in z_H^G (G = 2 where V has a
// parity); the groups' prefixes (the other variables and z_H^j0) form a trie
// over non-decreasing variable sequences, walked depth first (each prefix its
// parent times one variable), and a group's entries are the coefficients of
// (z_H^G)^0, (z_H^G)^1, .. (Horner in z_H^G; missing powers are zero entries).
constexpr int kNdMaxDim = 4;
constexpr int kNdMaxP = 12;
constexpr int kNdMaxDeg = 6;
constexpr int kNdMaxTerms = 256;
constexpr int kNdMaxDepth = 32;

struct NdEffective {
    int d = 0, p = 0, H = 0, G = 1;                     // Horner in z_H^G
    std::vector<int> depth, sym, first, count;          // depth-first nodes; node 0 = the empty prefix
    std::vector<std::vector<double>> hi, lo;            // entry -> coefficient of eps^q, q = 0..p-1
    std::vector<std::vector<unsigned char>> mono;       // entry -> exponents of z (2d)
};

int build_nd(int d, const int *exps, const double *coefs, int n_terms, int p, NdEffective &E, std::string &err);

// The level table for one eps: entry e gets -eps * sum_q c_q eps^q.
void nd_table(const NdEffective &E, double eps, std::vector<double> &T);

// W(x, xb; eps) on the host (level 0 and checks): x, xb of d entries.
double nd_wp_host(const NdEffective &E, const double *x, const double *xb, double eps);
// The same at n points, x and xb laid out [point][d], the table made once.
void nd_wp_points(const NdEffective &E, double eps, const double *x, const double *xb, int64_t n, double *w);

}  // namespace su
