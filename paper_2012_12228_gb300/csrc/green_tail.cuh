// The last step of the mixed-path Green kernels, run by one thread per walker
// once G(tau_k) and ln det M_k are known: ln det(I + A_k), the mu tangent
// k dtau (M - tr G) and the weight update of the chosen constraint.
#pragma once
#include <cmath>

#include "complex_math.cuh"
#include "ftq_internal.h"

namespace ftq {

// s: this walker's state row; ldm = sum of log pivots of M_k; lsum = sum of
// the logs of the two-sided scale factors split off before the factorisation;
// nswap = parity of the pivot permutation; trg = tr G(tau_k); kdt = k dtau.
__device__ __forceinline__ void green_weight_tail(double* s, double2 ldm, double lsum, int nswap, double2 trg, int M,
                                                  double kdt, int constraint, int* status) {
    constexpr double pi = 3.14159265358979323846;
    double2 ld = ldm;
    ld.x -= lsum;
    ld.y += pi * (double)(nswap ^ ((int)s[7]));
    if (!isfinite(ld.x) || !isfinite(ld.y)) atomicOr(status, 1);
    // d ln det(I + A_k)/dmu = k dtau (M - tr G(tau_k)): every B carries exp(dtau mu)
    const double2 tk = make_double2(kdt * ((double)M - trg.x), -kdt * trg.y);
    const double2 dlnS = make_double2(2.0 * (tk.x - s[9]), 2.0 * (tk.y - s[10]));
    const double2 lnS = make_double2(2.0 * (ld.x - s[3]), 2.0 * (ld.y - s[4]));
    const double gr = s[5], gi = s[6];
    if (constraint == FTQ_FREE) {
        s[0] += lnS.x + gr;
        s[1] = remainder(s[1] + lnS.y + gi, 2.0 * pi);
        s[8] += dlnS.x;
        s[11] += dlnS.y;
    } else if (s[2] > 0.5) {
        const double cth = cos(lnS.y);
        if (!isfinite(lnS.x + gr) || !(cth == cth)) {
            // a non-finite ratio or Gaussian factor drops the walker (weight 0)
            s[2] = 0.0;
            atomicOr(status, 1);
        } else if (cth <= 0.0) {
            s[2] = 0.0;
        } else {
            s[0] += lnS.x + gr + log(cth);
            s[8] += dlnS.x - tan(lnS.y) * dlnS.y;   // d log cos(theta) = -tan(theta) d theta
        }
    }
    s[3] = ld.x;
    s[4] = remainder(ld.y, 2.0 * pi);
    s[9] = tk.x;
    s[10] = tk.y;
}

}  // namespace ftq
