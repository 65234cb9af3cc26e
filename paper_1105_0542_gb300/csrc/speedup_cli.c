/* speedup -- the estimator from the command line, with the argument order of
 * the paper's program (Sec. 4): time of propagation T, endpoints a and b, the
 * deepest bisection level s, the number of Monte Carlo samples and the seed,
 * then the potential's parameters.  Prints the amplitude and its error for
 * every bisection level n = 0..s (level 0 is analytic, error 0).
 *
 * Plain C over the library's C ABI (include/speedup.h).
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "speedup.h"

static void usage(FILE *f) {
    fprintf(f,
            "usage: speedup [options] T a b s Nmc seed [par ...]\n"
            "  A_N^(p)(a, b; T) for N = 2^n, n = 0..s, from Nmc samples (seed), with the\n"
            "  level-p effective action of the model's potential V(q; par):\n"
            "    ho       omega^2 q^2 / 2                 par: omega\n"
            "    aho      A q^2/2 + g q^4/24              par: A g\n"
            "    dw       h (q^2 - 1)^2                   par: h\n"
            "    mpt      -lambda / cosh^2(alpha q)       par: lambda alpha\n"
            "    poly     sum_i v_i q^i (degree <= 8)     par: v_0 v_1 ...\n"
            "    general  polynomial + Gaussians + sech^2 (33 parameters, see speedup.h)\n"
            "options:\n"
            "  -m model     the potential (default aho)\n"
            "  -p level     effective-action level p (default 10)\n"
            "  -f fp64|fp32 precision of the path and W_p (default fp64)\n"
            "  -B blocks    contiguous sample blocks for the error (default 64)\n"
            "  -w factor    bisection width factor (default 1: the exact bridge)\n"
            "  -i instance  stream id (default 0)\n"
            "  -t           print the continuum fit A + B/N^p + C/N^(p+1) over N >= 8\n"
            "output: one line per level: n N amplitude error\n");
}

static int model_id(const char *s) {
    if (!strcmp(s, "ho")) return SU_HO;
    if (!strcmp(s, "aho")) return SU_AHO;
    if (!strcmp(s, "dw")) return SU_DW;
    if (!strcmp(s, "mpt")) return SU_MPT;
    if (!strcmp(s, "poly")) return SU_POLY;
    if (!strcmp(s, "general")) return SU_GENERAL;
    return -1;
}

static int num(const char *s, double *out) {
    char *end = NULL;
    *out = strtod(s, &end);
    return end != s && *end == '\0';
}

int main(int argc, char **argv) {
    if (argc < 2) {
        usage(stdout);
        return 0;
    }
    su_options o;
    su_options_default(&o);
    int model = SU_AHO, p = 10, fit = 0;
    int i = 1;
    for (; i < argc && argv[i][0] == '-' && argv[i][1] != '\0' && (argv[i][1] < '0' || argv[i][1] > '9') &&
           argv[i][1] != '.';
         ++i) {
        const char *opt = argv[i];
        if (!strcmp(opt, "-h") || !strcmp(opt, "--help")) {
            usage(stdout);
            return 0;
        }
        if (!strcmp(opt, "-t")) {
            fit = 1;
            continue;
        }
        if (i + 1 >= argc) {
            fprintf(stderr, "speedup: %s needs a value\n", opt);
            return 2;
        }
        const char *v = argv[++i];
        double x = 0;
        if (!strcmp(opt, "-m")) {
            if ((model = model_id(v)) < 0) {
                fprintf(stderr, "speedup: unknown model %s\n", v);
                return 2;
            }
        } else if (!strcmp(opt, "-f")) {
            if (!strcmp(v, "fp64")) o.precision = SU_FP64;
            else if (!strcmp(v, "fp32")) o.precision = SU_FP32;
            else {
                fprintf(stderr, "speedup: precision must be fp64 or fp32\n");
                return 2;
            }
        } else if (num(v, &x) && (!strcmp(opt, "-p") || !strcmp(opt, "-B") || !strcmp(opt, "-w") ||
                                  !strcmp(opt, "-i"))) {
            if (!strcmp(opt, "-p")) p = (int)x;
            if (!strcmp(opt, "-B")) o.n_blocks = (int)x;
            if (!strcmp(opt, "-w")) o.width_factor = x;
            if (!strcmp(opt, "-i")) o.instance = (uint32_t)x;
        } else {
            fprintf(stderr, "speedup: bad option %s %s\n", opt, v);
            return 2;
        }
    }
    if (argc - i < 6) {
        usage(stderr);
        return 2;
    }
    double T, a, b, sd, nd, seedd;
    if (!num(argv[i], &T) || !num(argv[i + 1], &a) || !num(argv[i + 2], &b) || !num(argv[i + 3], &sd) ||
        !num(argv[i + 4], &nd) || !num(argv[i + 5], &seedd)) {
        fprintf(stderr, "speedup: T a b s Nmc seed must be numbers\n");
        return 2;
    }
    const int s = (int)sd;
    const int npar = argc - i - 6;
    double par[64];
    if (npar > 64) {
        fprintf(stderr, "speedup: at most 64 potential parameters\n");
        return 2;
    }
    for (int k = 0; k < npar; ++k)
        if (!num(argv[i + 6 + k], &par[k])) {
            fprintf(stderr, "speedup: parameter %s is not a number\n", argv[i + 6 + k]);
            return 2;
        }
    if (s < 0 || s > SU_MAX_S) {
        fprintf(stderr, "speedup: s must be in 0..%d\n", SU_MAX_S);
        return 2;
    }
    su_level_result out[SU_MAX_S + 1];
    const int rc = speedup_amplitude(model, par, npar, a, b, T, p, s, (int64_t)nd, (uint64_t)seedd, &o, out);
    if (rc != SU_OK) {
        fprintf(stderr, "speedup: %s (code %d)\n", su_last_error(), rc);
        return 1;
    }
    for (int n = 0; n <= s; ++n) printf("%d %lld %.17g %.6g\n", n, 1LL << n, out[n].amp, out[n].err);
    if (fit && s >= 5) {
        double A = 0, dA = 0, chi2 = 0;
        if (su_fit_continuum(out, s, p, 3, 3, &A, &dA, &chi2) == SU_OK)
            printf("# continuum fit (N >= 8): %.17g +- %.6g (chi2 %.3g)\n", A, dA, chi2);
    }
    return 0;
}
