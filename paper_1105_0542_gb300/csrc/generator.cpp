// Host generator of the level-p effective potential W_p (Sec. 2.1 and 3.3).
//
// The recursion Eq. 1Drec,
//   8(m+k+1) c_{m,k} = (2k+2)(2k+1) c_{m,k+1} + c''_{m-1,k}
//                      - sum_{l=0}^{m-2} sum_r c'_{l,r} c'_{m-l-2,k-r}
//                      - sum_{l=1}^{m-2} sum_r 2r(2k-2r+2) c_{l,r} c_{m-l-1,k-r+1},
//   r in [max(0, k-m+l+2), min(k, l)],
// with c_{m,m} = V^(2m)/(2m+1)! (Eq. diagonal), evaluated for each m diagonal
// first and then k = m-1..0 (Fig. 1), on polynomials in one ring variable:
//
//  * x itself for polynomial potentials (the model-specific mode of Sec. 3.3:
//    derivatives taken explicitly while iterating);
//  * s = tanh^2(alpha x) for V = -lambda/cosh^2(alpha x) = -lambda (1 - s)
//    (Eq. 1D-MPT).  With t = tanh(alpha x), dt/dx = alpha (1 - t^2), so
//    ds/dx = 2 alpha t (1 - s), (ds/dx)^2 = 4 alpha^2 s (1-s)^2 and
//    d2s/dx2 = 2 alpha^2 (1-s)(1-3s):
//      f'(x) g'(x) = 4 alpha^2 s (1-s)^2 f_s g_s,
//      f''(x)      = 4 alpha^2 s (1-s)^2 f_ss + 2 alpha^2 (1-s)(1-3s) f_s,
//    and every c_{m,k} stays a polynomial in s (the content of
//    Eq. 1D-MPTansatz: tanh^(2l) / cosh^(2m-2l+2) = s^l (1-s)^(m-l+1)).
//    The basis s^i is chosen over powers of 1/cosh^2 = 1 - s because the
//    latter alternate in sign with binomial growth and lose digits in
//    single precision at large eps.
//
// Coefficients are double-double numbers (a + b with |b| <= ulp(a)/2, using
// Knuth's two-sum and the FMA-exact product), so that the collapse of many
// terms of alternating sign at large eps still rounds to double correctly.
// This file is host code; it is compiled with floating-point contraction off
// so that the error-free transformations stay error-free on every host.
#include "generator.h"

#include <algorithm>
#include <array>
#include <climits>
#include <cstdint>
#include <cmath>
#include <map>
#include <cstdio>

#include "../../include/speedup.h"

namespace su {
namespace {

struct DD {
    double hi, lo;
};

inline DD two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
inline DD fast_two_sum(double a, double b) {
    double s = a + b;
    return {s, b - (s - a)};
}
inline DD two_prod(double a, double b) {
    double p = a * b;
    return {p, std::fma(a, b, -p)};
}
inline DD add(DD a, DD b) {
    DD s = two_sum(a.hi, b.hi);
    DD t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}
inline DD neg(DD a) { return {-a.hi, -a.lo}; }
inline DD mul(DD a, DD b) {
    DD p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return fast_two_sum(p.hi, p.lo);
}
inline DD mul_d(DD a, double b) {
    DD p = two_prod(a.hi, b);
    p.lo += a.lo * b;
    return fast_two_sum(p.hi, p.lo);
}
inline DD div_d(DD a, double b) {
    double q1 = a.hi / b;
    DD r = add(a, neg(two_prod(q1, b)));
    double q2 = r.hi / b;
    DD q = fast_two_sum(q1, q2);
    r = add(r, neg(two_prod(q2, b)));
    return add(q, DD{r.hi / b, 0.0});
}
inline DD dd(double a) { return {a, 0.0}; }
inline bool is_zero(DD a) { return a.hi == 0.0 && a.lo == 0.0; }

using Poly = std::vector<DD>;

void trim(Poly &a) {
    while (!a.empty() && is_zero(a.back())) a.pop_back();
}
Poly padd(const Poly &a, const Poly &b) {
    Poly r(std::max(a.size(), b.size()), dd(0));
    for (size_t i = 0; i < a.size(); ++i) r[i] = add(r[i], a[i]);
    for (size_t i = 0; i < b.size(); ++i) r[i] = add(r[i], b[i]);
    trim(r);
    return r;
}
Poly pscale(const Poly &a, DD s) {
    Poly r(a.size());
    for (size_t i = 0; i < a.size(); ++i) r[i] = mul(a[i], s);
    trim(r);
    return r;
}
Poly pmul(const Poly &a, const Poly &b) {
    if (a.empty() || b.empty()) return {};
    Poly r(a.size() + b.size() - 1, dd(0));
    for (size_t i = 0; i < a.size(); ++i) {
        if (is_zero(a[i])) continue;
        for (size_t j = 0; j < b.size(); ++j)
            if (!is_zero(b[j])) r[i + j] = add(r[i + j], mul(a[i], b[j]));
    }
    trim(r);
    return r;
}
Poly pder(const Poly &a) {
    Poly r;
    for (size_t i = 1; i < a.size(); ++i) r.push_back(mul_d(a[i], (double)i));
    trim(r);
    return r;
}
// multiply by the monomial-sum sum_i m[i] u^i (small exact coefficients)
Poly pmul_small(const Poly &a, const Poly &m) { return pmul(a, m); }

// The ring: how x-derivatives act on the ring variable.
struct RingOps {
    bool tanh2 = false;
    Poly w;   // 4 alpha^2 s (1-s)^2: the factor of products of first derivatives
    Poly g;   // 2 alpha^2 (1-s)(1-3s): the factor of f_s in f''
    // first derivative in the ring variable (x or s)
    Poly d1(const Poly &f) const { return pder(f); }
    // x-second derivative
    Poly d2(const Poly &f) const {
        if (!tanh2) return pder(pder(f));
        return padd(pmul_small(pder(pder(f)), w), pmul_small(pder(f), g));
    }
    // sum of products of two x-first-derivatives, given the sum of the
    // products of their ring derivatives
    Poly finish_products(const Poly &s) const { return tanh2 ? pmul_small(s, w) : s; }
};

}  // namespace

int build_effective(int model, const double *params, int n_params, int p, Effective &E,
                    std::string &err) {
    auto bad = [&](const char *m) {
        err = m;
        return SU_EINVAL;
    };
    if (p < 1 || p > SU_MAX_P) return bad("p must be in 1..144");
    if (n_params < 0 || (n_params > 0 && !params)) return bad("params missing");
    for (int i = 0; i < n_params; ++i)
        if (!std::isfinite(params[i])) return bad("non-finite potential parameter");
    Poly V;
    RingOps R;
    double alpha = 0;
    switch (model) {
        case SU_HO:
            if (n_params != 1) return bad("SU_HO takes 1 parameter (omega)");
            V = {dd(0), dd(0), div_d(two_prod(params[0], params[0]), 2.0)};
            break;
        case SU_AHO:
            if (n_params != 2) return bad("SU_AHO takes 2 parameters (A, g)");
            V = {dd(0), dd(0), div_d(dd(params[0]), 2.0), dd(0), div_d(dd(params[1]), 24.0)};
            break;
        case SU_DW:
            if (n_params != 1) return bad("SU_DW takes 1 parameter (h)");
            V = {dd(params[0]), dd(0), mul_d(dd(params[0]), -2.0), dd(0), dd(params[0])};
            break;
        case SU_MPT: {
            if (n_params != 2) return bad("SU_MPT takes 2 parameters (lambda, alpha)");
            if (params[1] == 0.0) return bad("SU_MPT needs alpha != 0");
            alpha = params[1];
            V = {dd(-params[0]), dd(params[0])};      // -lambda (1 - s)
            DD a2 = two_prod(alpha, alpha);
            DD a4 = mul_d(a2, 4.0), a2x2 = mul_d(a2, 2.0);
            R.tanh2 = true;
            // 4 a^2 s (1 - 2s + s^2) and 2 a^2 (1 - 4s + 3s^2)
            R.w = {dd(0), a4, mul_d(a4, -2.0), a4};
            R.g = {a2x2, mul_d(a2x2, -4.0), mul_d(a2x2, 3.0)};
            break;
        }
        case SU_POLY:
            if (n_params < 1 || n_params > 9) return bad("SU_POLY takes 1..9 coefficients");
            for (int i = 0; i < n_params; ++i) V.push_back(dd(params[i]));
            break;
        default:
            return bad("unknown model");
    }
    trim(V);

    // x-derivatives of V of even order for the diagonal
    std::vector<Poly> V2(p);
    V2[0] = V;
    for (int m = 1; m < p; ++m) V2[m] = R.d2(V2[m - 1]);

    std::vector<std::vector<Poly>> c(p, std::vector<Poly>(p));
    std::vector<std::vector<Poly>> cu(p, std::vector<Poly>(p));  // ring first derivatives
    DD inv_fact = dd(1.0);  // 1/(2m+1)!, one exact-integer division at a time
    for (int m = 0; m < p; ++m) {
        if (m > 0) inv_fact = div_d(div_d(inv_fact, 2.0 * m), 2.0 * m + 1.0);
        c[m][m] = pscale(V2[m], inv_fact);
        cu[m][m] = R.d1(c[m][m]);
        for (int k = m - 1; k >= 0; --k) {
            Poly acc = pscale(c[m][k + 1], dd((double)((2 * k + 2) * (2 * k + 1))));
            acc = padd(acc, R.d2(c[m - 1][k]));
            Poly prod;
            for (int l = 0; l <= m - 2; ++l)
                for (int r = std::max(0, k - m + l + 2); r <= std::min(k, l); ++r)
                    prod = padd(prod, pmul(cu[l][r], cu[m - l - 2][k - r]));
            acc = padd(acc, pscale(R.finish_products(prod), dd(-1.0)));
            for (int l = 1; l <= m - 2; ++l)
                for (int r = std::max(0, k - m + l + 2); r <= std::min(k, l); ++r) {
                    int fac = 2 * r * (2 * k - 2 * r + 2);
                    if (fac) acc = padd(acc, pscale(pmul(c[l][r], c[m - l - 1][k - r + 1]), dd(-(double)fac)));
                }
            c[m][k] = pscale(acc, div_d(dd(1.0), 8.0 * (m + k + 1)));
            cu[m][k] = R.d1(c[m][k]);
        }
    }

    // shape of the collapsed polynomial
    bool even = !R.tanh2;
    for (int m = 0; m < p && even; ++m)
        for (int k = 0; k <= m && even; ++k)
            for (size_t i = 1; i < c[m][k].size(); i += 2)
                if (!is_zero(c[m][k][i])) even = false;
    Shape S;
    S.ring = R.tanh2 ? RING_TANH2 : (even ? RING_EVEN : RING_X);
    S.alpha = alpha;
    int ncol = 0;
    std::vector<int> len(p, 0);
    for (int k = 0; k < p; ++k) {
        int deg = -1;
        for (int m = k; m < p; ++m) deg = std::max(deg, (int)c[m][k].size() - 1);
        if (deg >= 0) {
            len[k] = (S.ring == RING_EVEN ? deg / 2 : deg) + 1;
            ncol = k + 1;
        }
    }
    if (ncol == 0) {  // V = 0: keep one (zero) entry so the table is never empty
        ncol = 1;
        len[0] = 1;
    }
    for (int k = 0; k < ncol; ++k)
        if (len[k] == 0) len[k] = 1;  // interior empty column: one zero entry
    S.ncol = ncol;
    S.len.assign(len.begin(), len.begin() + ncol);
    S.M = 0;
    for (int k = 0; k < ncol; ++k) S.M += S.len[k];

    E.p = p;
    E.shape = S;
    E.hi.assign(p, std::vector<std::vector<double>>(p));
    E.lo.assign(p, std::vector<std::vector<double>>(p));
    for (int m = 0; m < p; ++m)
        for (int k = 0; k <= m; ++k)
            for (const DD &v : c[m][k]) {
                E.hi[m][k].push_back(v.hi);
                E.lo[m][k].push_back(v.lo);
            }
    return SU_OK;
}

namespace {

// P_ij(eps) in double-double; ratio = sum|terms| / |sum| (largest)
void collapse_dd(const Effective &E, double eps, std::vector<DD> &P, double *ratio) {
    const Shape &S = E.shape;
    P.assign(S.M, dd(0));
    std::vector<DD> absum(S.M, dd(0));
    int off = 0;
    for (int j = 0; j < S.ncol; ++j) {
        DD ep = dd(1.0);  // eps^(m-j)
        for (int m = j; m < E.p; ++m) {
            const auto &h = E.hi[m][j];
            const auto &l = E.lo[m][j];
            for (size_t i = 0; i < h.size(); ++i) {
                if (S.ring == RING_EVEN && (i & 1)) continue;
                int ii = S.ring == RING_EVEN ? (int)i / 2 : (int)i;
                DD t = mul(DD{h[i], l[i]}, ep);
                P[off + ii] = add(P[off + ii], t);
                absum[off + ii] = add(absum[off + ii], DD{std::fabs(t.hi), std::fabs(t.hi) == t.hi ? t.lo : -t.lo});
            }
            ep = mul_d(ep, eps);
        }
        off += S.len[j];
    }
    if (ratio) {
        double r = 1.0;
        for (int i = 0; i < S.M; ++i)
            if (P[i].hi != 0.0) r = std::max(r, absum[i].hi / std::fabs(P[i].hi));
        *ratio = r;
    }
}

}  // namespace

void collapse(const Effective &E, double eps, std::vector<double> &P) {
    std::vector<DD> Pd;
    collapse_dd(E, eps, Pd, nullptr);
    P.resize(Pd.size());
    for (size_t i = 0; i < Pd.size(); ++i) P[i] = Pd[i].hi;
}

double kernel_table(const Effective &E, double eps, std::vector<double> &T) {
    std::vector<DD> Pd;
    double ratio = 1.0;
    collapse_dd(E, eps, Pd, &ratio);
    const Shape &S = E.shape;
    T.resize(S.M);
    int off = 0;
    for (int j = 0; j < S.ncol; ++j) {
        double sj = std::ldexp(1.0, -2 * j);  // xb^(2j) = vs^(2j) / 4^j
        for (int i = 0; i < S.len[j]; ++i) {
            double si = S.ring == RING_EVEN ? std::ldexp(1.0, -2 * i)    // x^(2i) = us^(2i)/4^i
                        : S.ring == RING_X  ? std::ldexp(1.0, -i)        // x^i = us^i / 2^i
                                            : 1.0;
            DD v = mul_d(mul_d(Pd[off + i], -eps), si * sj);  // powers of two: exact
            T[off + i] = v.hi;
        }
        off += S.len[j];
    }
    return ratio;
}

static double wp_from_dd(const Shape &S, const std::vector<DD> &Pd, double x, double xb) {
    double z = S.ring == RING_EVEN ? x * x
               : S.ring == RING_X  ? x
                                   : std::tanh(S.alpha * x) * std::tanh(S.alpha * x);
    DD y = two_prod(xb, xb);
    DD acc = dd(0);
    int off = S.M;
    for (int j = S.ncol - 1; j >= 0; --j) {
        off -= S.len[j];
        DD h = dd(0);
        for (int i = S.len[j] - 1; i >= 0; --i) h = add(mul_d(h, z), Pd[off + i]);
        acc = add(mul(acc, y), h);
    }
    return acc.hi;
}

double wp_host(const Effective &E, double x, double xb, double eps) {
    std::vector<DD> Pd;
    collapse_dd(E, eps, Pd, nullptr);
    return wp_from_dd(E.shape, Pd, x, xb);
}

void wp_host_points(const Effective &E, double eps, const double *x, const double *xb, int64_t n, double *w) {
    std::vector<DD> Pd;
    collapse_dd(E, eps, Pd, nullptr);
    for (int64_t i = 0; i < n; ++i) w[i] = wp_from_dd(E.shape, Pd, x[i], xb[i]);
}

double wp_collapsed(const Shape &S, const std::vector<double> &P, double x, double xb) {
    const double z = S.ring == RING_EVEN ? x * x
                     : S.ring == RING_X  ? x
                                         : std::tanh(S.alpha * x) * std::tanh(S.alpha * x);
    const double y = xb * xb;
    double acc = 0;
    int off = S.M;
    for (int j = S.ncol - 1; j >= 0; --j) {
        off -= S.len[j];
        double h = 0;
        for (int i = S.len[j] - 1; i >= 0; --i) h = h * z + P[off + i];
        acc = acc * y + h;
    }
    return acc;
}

// ---------------------------------------------------- general potentials
namespace {

using Mono = std::vector<unsigned char>;   // exponents of V_0..V_{2p-1}
using GPoly = std::map<Mono, DD>;

// acc += s * b, dropping sums that cancel to rounding residue
void gadd(GPoly &acc, const GPoly &b, DD s) {
    for (const auto &kv : b) {
        const DD v = mul(kv.second, s);
        auto it = acc.find(kv.first);
        if (it == acc.end()) {
            acc.emplace(kv.first, v);
        } else {
            const double scale = std::max(std::fabs(it->second.hi), std::fabs(v.hi));
            it->second = add(it->second, v);
            if (std::fabs(it->second.hi) <= 1e-26 * scale) acc.erase(it);
        }
    }
}

GPoly gmul(const GPoly &a, const GPoly &b) {
    GPoly out;
    for (const auto &x : a)
        for (const auto &y : b) {
            Mono m(x.first.size());
            for (size_t j = 0; j < m.size(); ++j) m[j] = (unsigned char)(x.first[j] + y.first[j]);
            GPoly t;
            t.emplace(std::move(m), mul(x.second, y.second));
            gadd(out, t, dd(1.0));
        }
    return out;
}

// d/dx with d/dx V_j = V_{j+1}
GPoly gD(const GPoly &a) {
    GPoly out;
    for (const auto &x : a)
        for (size_t j = 0; j + 1 < x.first.size(); ++j) {
            if (!x.first[j]) continue;
            Mono m = x.first;
            m[j] -= 1;
            m[j + 1] += 1;
            GPoly t;
            t.emplace(std::move(m), mul_d(x.second, (double)x.first[j]));
            gadd(out, t, dd(1.0));
        }
    return out;
}

}  // namespace

int build_general(int p, GeneralEffective &G, std::string &err) {
    if (p < 1 || p > kGenMaxP) {
        err = "the general potential supports p in 1..18";
        return SU_EINVAL;
    }
    const int nsym = 2 * p;   // V_0..V_{2p-1}; W_p uses up to V_{2p-2}
    std::vector<std::vector<GPoly>> c(p, std::vector<GPoly>(p)), dc(p, std::vector<GPoly>(p));
    DD inv_fact = dd(1.0);
    for (int m = 0; m < p; ++m) {
        if (m > 0) inv_fact = div_d(div_d(inv_fact, 2.0 * m), 2.0 * m + 1.0);
        Mono e(nsym, 0);
        e[2 * m] = 1;
        c[m][m].emplace(e, inv_fact);
        dc[m][m] = gD(c[m][m]);
        for (int k = m - 1; k >= 0; --k) {
            GPoly acc;
            gadd(acc, c[m][k + 1], dd((double)((2 * k + 2) * (2 * k + 1))));
            gadd(acc, gD(dc[m - 1][k]), dd(1.0));
            for (int l = 0; l <= m - 2; ++l)
                for (int r = std::max(0, k - m + l + 2); r <= std::min(k, l); ++r)
                    gadd(acc, gmul(dc[l][r], dc[m - l - 2][k - r]), dd(-1.0));
            for (int l = 1; l <= m - 2; ++l)
                for (int r = std::max(0, k - m + l + 2); r <= std::min(k, l); ++r) {
                    const int fac = 2 * r * (2 * k - 2 * r + 2);
                    if (fac) gadd(acc, gmul(c[l][r], c[m - l - 1][k - r + 1]), dd(-(double)fac));
                }
            GPoly ck;
            gadd(ck, acc, div_d(dd(1.0), 8.0 * (m + k + 1)));
            c[m][k] = std::move(ck);
            if (m < p - 1) dc[m][k] = gD(c[m][k]);
        }
    }
    // monomial -> per k: coefficients of eps^(m-k), m = k..p-1
    std::map<Mono, std::map<int, std::vector<DD>>> terms;
    int K = 1;
    for (int m = 0; m < p; ++m)
        for (int k = 0; k <= m; ++k)
            for (const auto &kv : c[m][k]) {
                auto &vec = terms[kv.first][k];
                if (vec.empty()) vec.assign((size_t)(p - k), dd(0));
                vec[(size_t)(m - k)] = kv.second;
                K = std::max(K, k + 1);
            }
    // trie over non-decreasing symbol sequences, children ordered by symbol
    struct TNode {
        std::map<int, int> child;
        const std::map<int, std::vector<DD>> *entries = nullptr;
    };
    std::vector<TNode> trie(1);
    for (const auto &kv : terms) {
        int node = 0;
        for (int j = 0; j < nsym; ++j)
            for (int r = 0; r < kv.first[(size_t)j]; ++r) {
                auto it = trie[(size_t)node].child.find(j);
                if (it == trie[(size_t)node].child.end()) {
                    trie.emplace_back();
                    const int nn = (int)trie.size() - 1;
                    trie[(size_t)node].child.emplace(j, nn);
                    node = nn;
                } else {
                    node = it->second;
                }
            }
        trie[(size_t)node].entries = &kv.second;
    }
    G = GeneralEffective{};
    G.p = p;
    G.J = std::max(2 * p - 2, 0);
    G.K = K;
    // depth-first, pre-order
    struct Frame {
        int node, depth, sym;
    };
    std::vector<Frame> stack{{0, 0, -1}};
    while (!stack.empty()) {
        const Frame f = stack.back();
        stack.pop_back();
        G.depth.push_back(f.depth);
        G.sym.push_back(std::max(f.sym, 0));
        G.first.push_back((int)G.entry_k.size());
        int cnt = 0;
        if (trie[(size_t)f.node].entries)
            for (const auto &e : *trie[(size_t)f.node].entries) {
                G.entry_k.push_back(e.first);
                std::vector<double> hi, lo;
                for (const DD &v : e.second) {
                    hi.push_back(v.hi);
                    lo.push_back(v.lo);
                }
                G.entry_hi.push_back(std::move(hi));
                G.entry_lo.push_back(std::move(lo));
                ++cnt;
            }
        G.count.push_back(cnt);
        const auto &ch = trie[(size_t)f.node].child;
        for (auto it = ch.rbegin(); it != ch.rend(); ++it) stack.push_back({it->second, f.depth + 1, it->first});
    }
    for (int s2 : G.sym)
        if (s2 > G.J) {
            err = "internal: a symbol beyond V^(2p-2) in W_p";
            return SU_EINVAL;
        }
    return SU_OK;
}

void general_table(const GeneralEffective &G, double eps, std::vector<double> &T) {
    T.resize(G.entry_k.size());
    for (size_t e = 0; e < G.entry_k.size(); ++e) {
        const int k = G.entry_k[e];
        DD acc = dd(0), pw = dd(1.0);
        for (size_t q = 0; q < G.entry_hi[e].size(); ++q) {   // eps^(m-k), m = k + q
            acc = add(acc, mul(DD{G.entry_hi[e][q], G.entry_lo[e][q]}, pw));
            pw = mul_d(pw, eps);
        }
        T[e] = mul_d(mul_d(acc, -eps), std::ldexp(1.0, -2 * k)).hi;
    }
}

int general_potential(const double *params, int n_params, GeneralPotential &V, std::string &err) {
    if ((n_params != kGenParams && n_params != kGenParamsExp) || !params) {
        err = "SU_GENERAL takes 33 parameters (a_0..a_8, (A, beta, c) x 4, (B, alpha, d) x 4) or 45 "
              "(then (E, kappa, x0) x 4)";
        return SU_EINVAL;
    }
    for (int i = 0; i < n_params; ++i)
        if (!std::isfinite(params[i])) {
            err = "non-finite potential parameter";
            return SU_EINVAL;
        }
    V = GeneralPotential{};
    for (int i = 0; i < 9; ++i) V.a[i] = params[i];
    for (int g = 0; g < 4; ++g) {
        const double *q = params + 9 + 3 * g;
        if (q[0] == 0.0) continue;
        if (!(q[1] > 0)) {
            err = "a Gaussian term needs beta > 0";
            return SU_EINVAL;
        }
        for (int r = 0; r < 3; ++r) V.gauss[V.ng][r] = q[r];
        ++V.ng;
    }
    for (int t = 0; t < 4; ++t) {
        const double *q = params + 21 + 3 * t;
        if (q[0] == 0.0) continue;
        if (q[1] == 0.0) {
            err = "a sech^2 term needs alpha != 0";
            return SU_EINVAL;
        }
        for (int r = 0; r < 3; ++r) V.sech[V.ns][r] = q[r];
        ++V.ns;
    }
    for (int t = 0; n_params == kGenParamsExp && t < 4; ++t) {
        const double *q = params + kGenParams + 3 * t;
        if (q[0] == 0.0) continue;
        for (int r = 0; r < 3; ++r) V.expo[V.ne][r] = q[r];
        ++V.ne;
    }
    return SU_OK;
}

void general_derivatives(const GeneralPotential &V, double x, int J, double *out) {
    for (int j = 0; j <= J; ++j) {
        double v = 0.0;   // sum_{i>=j} a_i i!/(i-j)! x^(i-j)
        for (int i = 8; i >= j; --i) {
            double f = 1.0;
            for (int r = 0; r < j; ++r) f *= (double)(i - r);
            v = v * x + V.a[i] * f;
        }
        out[j] = j <= 8 ? v : 0.0;
    }
    for (int g = 0; g < V.ng; ++g) {
        const double A = V.gauss[g][0], beta = V.gauss[g][1], c = V.gauss[g][2];
        const double sb = std::sqrt(beta), u = x - c, y = sb * u, e = A * std::exp(-beta * u * u);
        double h0 = 1.0, h1 = 2.0 * y, f = 1.0;
        for (int n = 0; n <= J; ++n) {
            const double h = n == 0 ? h0 : h1;
            out[n] += f * h * e;
            f *= -sb;
            if (n >= 1) {
                const double h2 = 2.0 * y * h1 - 2.0 * n * h0;
                h0 = h1;
                h1 = h2;
            }
        }
    }
    // sech^2 = tanh': Taylor coefficients a_k of tanh at alpha (x - d),
    // (n+1) a_{n+1} = -sum_k a_k a_{n-k} (n >= 1) from tanh' = 1 - tanh^2
    std::vector<double> a((size_t)J + 2);
    for (int s = 0; s < V.ns; ++s) {
        const double B = V.sech[s][0], alpha = V.sech[s][1], d = V.sech[s][2];
        const double w = alpha * (x - d), ch = std::cosh(w);
        a[0] = std::tanh(w);
        a[1] = 1.0 / (ch * ch);
        double sc = B;   // B alpha^n (n+1)!
        for (int n = 0; n <= J; ++n) {
            if (n >= 1) {
                double acc = 0.0;
                for (int k = 0; k <= n; ++k) acc += a[(size_t)k] * a[(size_t)(n - k)];
                a[(size_t)n + 1] = -acc / (double)(n + 1);
            }
            sc *= (double)(n + 1);
            out[n] += sc * a[(size_t)n + 1];
            sc *= alpha;
        }
    }
    // exponentials: (-kappa)^n E e^{-kappa (x - x0)}
    for (int t = 0; t < V.ne; ++t) {
        double e = V.expo[t][0] * std::exp(-V.expo[t][1] * (x - V.expo[t][2]));
        for (int n = 0; n <= J; ++n) {
            out[n] += e;
            e *= -V.expo[t][1];
        }
    }
}

static double general_wp_from_table(const GeneralEffective &G, const GeneralPotential &V,
                                    const std::vector<double> &T, double x, double xb, double eps) {
    std::vector<double> D((size_t)G.J + 1);
    general_derivatives(V, x, G.J, D.data());
    std::vector<double> stk((size_t)G.J + 3 * G.p + 2, 1.0), Q((size_t)G.K, 0.0);
    for (size_t t = 0; t < G.depth.size(); ++t) {
        double mu = 1.0;
        if (t) {
            mu = stk[(size_t)G.depth[t] - 1] * D[(size_t)G.sym[t]];
            stk[(size_t)G.depth[t]] = mu;
        }
        for (int e = G.first[t]; e < G.first[t] + G.count[t]; ++e) Q[(size_t)G.entry_k[(size_t)e]] += T[(size_t)e] * mu;
    }
    const double Y = 4.0 * xb * xb;   // vs^2
    double w = Q[(size_t)G.K - 1];
    for (int k = G.K - 2; k >= 0; --k) w = w * Y + Q[(size_t)k];
    return -w / eps;                  // the table carries -eps
}

double general_wp_host(const GeneralEffective &G, const GeneralPotential &V, double x, double xb, double eps) {
    std::vector<double> T;
    general_table(G, eps, T);   // -eps c / 4^k per entry
    return general_wp_from_table(G, V, T, x, xb, eps);
}

void general_wp_points(const GeneralEffective &G, const GeneralPotential &V, double eps, const double *x,
                       const double *xb, int64_t n, double *w) {
    std::vector<double> T;
    general_table(G, eps, T);
    for (int64_t i = 0; i < n; ++i) w[i] = general_wp_from_table(G, V, T, x[i], xb[i], eps);
}

// ------------------------------------------- systems of d coordinates
namespace {

using NM = std::array<unsigned char, 2 * kNdMaxDim>;   // exponents of x_1..x_d, xb_1..xb_d
using NPoly = std::map<NM, DD>;

// acc += s * b, dropping sums that cancel to rounding residue
void nadd(NPoly &acc, const NPoly &b, DD s) {
    for (const auto &kv : b) {
        const DD v = mul(kv.second, s);
        auto it = acc.find(kv.first);
        if (it == acc.end()) {
            acc.emplace(kv.first, v);
        } else {
            const double scale = std::max(std::fabs(it->second.hi), std::fabs(v.hi));
            it->second = add(it->second, v);
            if (std::fabs(it->second.hi) <= 1e-26 * scale) acc.erase(it);
        }
    }
}

void nadd_term(NPoly &acc, const NM &m, DD v) {
    auto it = acc.find(m);
    if (it == acc.end()) {
        acc.emplace(m, v);
    } else {
        const double scale = std::max(std::fabs(it->second.hi), std::fabs(v.hi));
        it->second = add(it->second, v);
        if (std::fabs(it->second.hi) <= 1e-26 * scale) acc.erase(it);
    }
}

NPoly nmul(const NPoly &a, const NPoly &b) {
    NPoly out;
    for (const auto &x : a)
        for (const auto &y : b) {
            NM m;
            for (size_t j = 0; j < m.size(); ++j) m[j] = (unsigned char)(x.first[j] + y.first[j]);
            nadd_term(out, m, mul(x.second, y.second));
        }
    return out;
}

// d/dz_i
NPoly nder(const NPoly &a, int i) {
    NPoly out;
    for (const auto &x : a) {
        if (!x.first[(size_t)i]) continue;
        NM m = x.first;
        m[(size_t)i] -= 1;
        nadd_term(out, m, mul_d(x.second, (double)x.first[(size_t)i]));
    }
    return out;
}

}  // namespace

int build_nd(int d, const int *exps, const double *coefs, int n_terms, int p, NdEffective &E, std::string &err) {
    if (d < 1 || d > kNdMaxDim) {
        err = "the dimension d = D x M must be in 1..4";
        return SU_EINVAL;
    }
    if (p < 1 || p > kNdMaxP) {
        err = "p must be in 1..12 for systems of several coordinates";
        return SU_EINVAL;
    }
    if (!exps || !coefs || n_terms < 1 || n_terms > kNdMaxTerms) {
        err = "the potential needs 1..256 terms";
        return SU_EINVAL;
    }
    NPoly V;
    for (int t = 0; t < n_terms; ++t) {
        NM m{};
        int deg = 0;
        for (int i = 0; i < d; ++i) {
            const int e = exps[t * d + i];
            if (e < 0 || e > kNdMaxDeg) {
                err = "potential exponents must be in 0..6";
                return SU_EINVAL;
            }
            m[(size_t)i] = (unsigned char)e;
            deg += e;
        }
        if (deg > kNdMaxDeg) {
            err = "the potential's total degree must be <= 6";
            return SU_EINVAL;
        }
        if (!std::isfinite(coefs[t])) {
            err = "non-finite potential coefficient";
            return SU_EINVAL;
        }
        if (coefs[t] != 0.0) nadd_term(V, m, dd(coefs[t]));
    }
    // W[m][k] and its gradients in x and in xb
    std::vector<std::vector<NPoly>> W((size_t)p, std::vector<NPoly>((size_t)p));
    std::vector<std::vector<std::vector<NPoly>>> gx((size_t)p, std::vector<std::vector<NPoly>>((size_t)p)),
        gb((size_t)p, std::vector<std::vector<NPoly>>((size_t)p));
    auto grads = [&](int m, int k) {
        gx[(size_t)m][(size_t)k].resize((size_t)d);
        gb[(size_t)m][(size_t)k].resize((size_t)d);
        for (int i = 0; i < d; ++i) {
            gx[(size_t)m][(size_t)k][(size_t)i] = nder(W[(size_t)m][(size_t)k], i);
            gb[(size_t)m][(size_t)k][(size_t)i] = nder(W[(size_t)m][(size_t)k], d + i);
        }
    };
    auto dot = [&](const std::vector<NPoly> &a, const std::vector<NPoly> &b, NPoly &acc, DD s) {
        for (int i = 0; i < d; ++i) nadd(acc, nmul(a[(size_t)i], b[(size_t)i]), s);
    };
    NPoly diag = V;   // (xb . grad)^(2m) V
    DD inv_fact = dd(1.0);
    for (int m = 0; m < p; ++m) {
        if (m > 0) {
            for (int rep = 0; rep < 2; ++rep) {
                NPoly nxt;
                for (int i = 0; i < d; ++i) {
                    NPoly t = nder(diag, i);
                    for (const auto &x : t) {
                        NM mm = x.first;
                        mm[(size_t)(d + i)] += 1;
                        nadd_term(nxt, mm, x.second);
                    }
                }
                diag = std::move(nxt);
            }
            inv_fact = div_d(div_d(inv_fact, 2.0 * m), 2.0 * m + 1.0);
        }
        NPoly &wmm = W[(size_t)m][(size_t)m];
        nadd(wmm, diag, inv_fact);
        grads(m, m);
        for (int k = m - 1; k >= 0; --k) {
            NPoly acc;
            for (int i = 0; i < d; ++i) {   // lap W_{m-1,k} + lapb W_{m,k+1}
                nadd(acc, nder(gx[(size_t)m - 1][(size_t)k][(size_t)i], i), dd(1.0));
                nadd(acc, nder(gb[(size_t)m][(size_t)k + 1][(size_t)i], d + i), dd(1.0));
            }
            for (int l = 0; l <= m - 2; ++l)
                for (int r = std::max(0, k - m + l + 2); r <= std::min(k, l); ++r)
                    dot(gx[(size_t)l][(size_t)r], gx[(size_t)(m - l - 2)][(size_t)(k - r)], acc, dd(-1.0));
            for (int l = 1; l <= m - 2; ++l)
                for (int r = std::max(0, k - m + l + 2); r <= std::min(k, l); ++r)
                    dot(gb[(size_t)l][(size_t)r], gb[(size_t)(m - l - 1)][(size_t)(k - r + 1)], acc, dd(-1.0));
            nadd(W[(size_t)m][(size_t)k], acc, div_d(dd(1.0), 8.0 * (m + k + 1)));
            grads(m, k);
        }
    }
    // monomial -> coefficient of eps^q, q = m - k
    std::map<NM, std::vector<DD>> terms;
    for (int m = 0; m < p; ++m)
        for (int k = 0; k <= m; ++k)
            for (const auto &kv : W[(size_t)m][(size_t)k]) {
                auto &v = terms[kv.first];
                if (v.empty()) v.assign((size_t)p, dd(0));
                v[(size_t)(m - k)] = add(v[(size_t)(m - k)], kv.second);
            }
    // the Horner variable z_H and step G: a group (the monomials that agree
    // in every other variable) is z_H^j0 sum_i c_i (z_H^G)^i, j0 its lowest
    // power of z_H, which joins the group's prefix; G is the gcd of the power
    // differences inside groups (2 where V has a parity).  Taken to make the
    // program shortest (trie nodes + entries).
    const int nv = 2 * d;
    auto others_of = [&](const NM &m, int H) {
        NM o = m;
        o[(size_t)H] = 0;
        return o;
    };
    auto seq_of = [&](const NM &o, int H, int j0) {
        std::vector<int> seq;
        for (int v = 0; v < nv; ++v) {
            const int reps = v == H ? j0 : (int)o[(size_t)v];
            for (int r = 0; r < reps; ++r) seq.push_back(v);
        }
        return seq;
    };
    struct Span {
        int lo = INT_MAX, hi = -1, g = 0;
    };
    auto spans_of = [&](int H, int &G) {
        std::map<NM, Span> grp;
        for (const auto &kv : terms) {
            Span &sp = grp[others_of(kv.first, H)];
            const int e = kv.first[(size_t)H];
            sp.lo = std::min(sp.lo, e);
            sp.hi = std::max(sp.hi, e);
        }
        G = 0;
        for (const auto &kv : terms) {
            const Span &sp = grp[others_of(kv.first, H)];
            int a = G, b = kv.first[(size_t)H] - sp.lo;
            while (b) {
                const int t = a % b;
                a = b;
                b = t;
            }
            G = a;
        }
        if (G == 0) G = 1;
        return grp;
    };
    int bestH = 0, bestG = 1;
    size_t best = SIZE_MAX;
    for (int H = 0; H < nv; ++H) {
        int G = 1;
        const auto grp = spans_of(H, G);
        std::map<std::vector<int>, int> trie;   // every prefix of every group's prefix
        size_t entries = 0;
        for (const auto &g : grp) {
            entries += (size_t)((g.second.hi - g.second.lo) / G + 1);
            const std::vector<int> seq = seq_of(g.first, H, g.second.lo);
            for (size_t len = 0; len <= seq.size(); ++len)
                trie.emplace(std::vector<int>(seq.begin(), seq.begin() + (long)len), 0);
        }
        if (trie.size() + entries < best) {
            best = trie.size() + entries;
            bestH = H;
            bestG = G;
        }
    }
    // the program: trie over prefixes, depth first, children by variable
    struct TNode {
        std::map<int, int> child;
        int imax = -1, j0 = 0;
        std::vector<std::vector<DD>> coef;   // power of z_H^G -> per-q coefficients
        std::vector<int> seq;
    };
    int G0 = 1;
    const auto groups = spans_of(bestH, G0);
    std::vector<TNode> trie(1);
    for (const auto &kv : terms) {
        const NM o = others_of(kv.first, bestH);
        const int j0 = groups.at(o).lo;
        const std::vector<int> seq = seq_of(o, bestH, j0);
        int node = 0;
        for (size_t t = 0; t < seq.size(); ++t) {
            auto it = trie[(size_t)node].child.find(seq[t]);
            if (it == trie[(size_t)node].child.end()) {
                trie.emplace_back();
                const int nn = (int)trie.size() - 1;
                trie[(size_t)nn].seq.assign(seq.begin(), seq.begin() + (long)t + 1);
                trie[(size_t)node].child.emplace(seq[t], nn);
                node = nn;
            } else {
                node = it->second;
            }
        }
        TNode &tn = trie[(size_t)node];
        tn.j0 = j0;
        const int i = (kv.first[(size_t)bestH] - j0) / bestG;
        if (i > tn.imax) {
            tn.coef.resize((size_t)i + 1, std::vector<DD>((size_t)p, dd(0)));
            tn.imax = i;
        }
        tn.coef[(size_t)i] = kv.second;
    }
    E = NdEffective{};
    E.d = d;
    E.p = p;
    E.H = bestH;
    E.G = bestG;
    struct Frame {
        int node, depth, sym;
    };
    std::vector<Frame> stack{{0, 0, -1}};
    while (!stack.empty()) {
        const Frame f = stack.back();
        stack.pop_back();
        if (f.depth > kNdMaxDepth) {
            err = "the effective potential's degree exceeds the evaluation program's depth (32)";
            return SU_ENOTSUP;
        }
        const TNode &tn = trie[(size_t)f.node];
        E.depth.push_back(f.depth);
        E.sym.push_back(std::max(f.sym, 0));
        E.first.push_back((int)E.hi.size());
        E.count.push_back(tn.imax + 1);
        for (int i = 0; i <= tn.imax; ++i) {
            std::vector<double> hi, lo;
            for (const DD &v : tn.coef[(size_t)i]) {
                hi.push_back(v.hi);
                lo.push_back(v.lo);
            }
            E.hi.push_back(std::move(hi));
            E.lo.push_back(std::move(lo));
            std::vector<unsigned char> mono((size_t)nv, 0);
            for (int v : tn.seq) mono[(size_t)v] += 1;   // includes z_H^j0
            mono[(size_t)bestH] = (unsigned char)(mono[(size_t)bestH] + bestG * i);
            E.mono.push_back(std::move(mono));
        }
        for (auto it = tn.child.rbegin(); it != tn.child.rend(); ++it) stack.push_back({it->second, f.depth + 1, it->first});
    }
    return SU_OK;
}

void nd_table(const NdEffective &E, double eps, std::vector<double> &T) {
    T.resize(E.hi.size());
    for (size_t e = 0; e < E.hi.size(); ++e) {
        DD acc = dd(0);
        for (size_t q = E.hi[e].size(); q-- > 0;) acc = add(mul_d(acc, eps), DD{E.hi[e][q], E.lo[e][q]});
        T[e] = mul_d(acc, -eps).hi;
    }
}

static double nd_wp_from_table(const NdEffective &E, const std::vector<double> &T, const double *x,
                               const double *xb, double eps) {
    double z[2 * kNdMaxDim];
    for (int i = 0; i < E.d; ++i) {
        z[i] = x[i];
        z[E.d + i] = xb[i];
    }
    double Y = 1.0;
    for (int g = 0; g < E.G; ++g) Y *= z[E.H];
    std::vector<double> stk((size_t)kNdMaxDepth + 1, 1.0);
    double w = 0.0;
    for (size_t t = 0; t < E.depth.size(); ++t) {
        double mu = 1.0;
        if (t) {
            mu = stk[(size_t)E.depth[t] - 1] * z[E.sym[t]];
            stk[(size_t)E.depth[t]] = mu;
        }
        if (!E.count[t]) continue;
        double h = T[(size_t)(E.first[t] + E.count[t] - 1)];
        for (int j = E.count[t] - 2; j >= 0; --j) h = h * Y + T[(size_t)(E.first[t] + j)];
        w += h * mu;
    }
    return -w / eps;   // the table carries -eps
}

double nd_wp_host(const NdEffective &E, const double *x, const double *xb, double eps) {
    std::vector<double> T;
    nd_table(E, eps, T);
    return nd_wp_from_table(E, T, x, xb, eps);
}

void nd_wp_points(const NdEffective &E, double eps, const double *x, const double *xb, int64_t n, double *w) {
    std::vector<double> T;
    nd_table(E, eps, T);
    for (int64_t i = 0; i < n; ++i) w[i] = nd_wp_from_table(E, T, x + i * E.d, xb + i * E.d, eps);
}

}  // namespace su
