// adaptive.cu -- the fault-coverage model and the per-step mode policy of
// adaptive ABFT (Sec. 3.1.2, Alg. alg-abft), on the host.  Errors of type 0D,
// 1D and 2D arrive as independent Poisson processes; in one detection
// interval of T seconds their counts are Poisson(lambda T) = Poisson(mu).
// The matrix has S blocks, each error strikes one uniformly at random, and a
// block corrects at most one error per interval.  Single-side checksums
// correct 0D errors only, full checksums 0D and 1D errors, neither 2D ones:
//   FC_single = [sum_k Pois(k; mu0) prod_{i<k} (S - i) / S] e^-mu1 e^-mu2
//   FC_full   = [sum_k sum_j Pois(k; mu0) Pois(j; mu1) prod_{i<k+j} (S-i)/S] e^-mu2
// The distinct-block product runs to k - 1 (k errors in k distinct blocks).
// FC_full is evaluated through the identity sum_{k+j=c} Pois(k; mu0)
// Pois(j; mu1) = Pois(c; mu0 + mu1), one sum instead of two.  Sums stop once
// the Poisson weights past the mode fall below 1e-300.
#include <math.h>
#include <stdint.h>

#include "abft.h"

namespace {

double covered(int64_t S, double mu) {
    if (!(mu > 0.0)) return 1.0;
    double t = exp(-mu), p = 1.0, sum = 0.0;
    for (int64_t k = 0; k <= S; ++k) {
        sum += t * p;
        p *= (double)(S - k) / (double)S;      // prod_{i<=k}: for the next term
        t *= mu / (double)(k + 1);
        if ((t < 1e-300 && (double)k > mu) || p == 0.0) break;
    }
    return sum;
}

}  // namespace

extern "C" {

double abft_fc_single(int64_t S, double mu0, double mu1, double mu2) {
    if (S <= 0 || !(mu0 >= 0.0) || !(mu1 >= 0.0) || !(mu2 >= 0.0)) return NAN;
    return covered(S, mu0) * exp(-mu1) * exp(-mu2);
}

double abft_fc_full(int64_t S, double mu0, double mu1, double mu2) {
    if (S <= 0 || !(mu0 >= 0.0) || !(mu1 >= 0.0) || !(mu2 >= 0.0)) return NAN;
    return covered(S, mu0 + mu1) * exp(-mu2);
}

int abft_adaptive_modes(int64_t n, int64_t nb, const double* lambda, double fc_desired,
                        const double* step_seconds, int32_t* modes, double* coverage) {
    if (n < 0) return -1;
    if (nb <= 0) return -2;
    if (lambda == nullptr || !(lambda[0] >= 0.0) || !(lambda[1] >= 0.0) || !(lambda[2] >= 0.0))
        return -3;
    if (!(fc_desired >= 0.0 && fc_desired <= 1.0)) return -4;
    const int64_t N = (n + nb - 1) / nb;
    if (N > 0 && (step_seconds == nullptr || modes == nullptr)) return -5;
    const int64_t S = N * N;
    for (int64_t k = 0; k < N; ++k) {
        const double T = step_seconds[k];
        if (!(T >= 0.0)) return -5;
        int32_t m;
        double c;
        if (lambda[0] == 0.0 && lambda[1] == 0.0 && lambda[2] == 0.0) {
            m = ABFT_MODE_NONE;
            c = 1.0;
        } else {
            c = abft_fc_single(S, lambda[0] * T, lambda[1] * T, lambda[2] * T);
            m = ABFT_MODE_SINGLE;
            if (!(c >= fc_desired)) {
                c = abft_fc_full(S, lambda[0] * T, lambda[1] * T, lambda[2] * T);
                m = ABFT_MODE_FULL;
            }
        }
        modes[k] = m;
        if (coverage) coverage[k] = c;
    }
    return ABFT_OK;
}

}  // extern "C"
