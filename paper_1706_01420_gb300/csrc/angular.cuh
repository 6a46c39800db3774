// The ten angular functions of the helicity basis (Sec. 4 and the
// symbolic-programming section: P wave and S wave of B_s -> J/psi K K), shared
// by the likelihood kernels of the 4D and the phi_s models and the basis
// kernel: f_k = c_k f'_k with f'_k a product of sines and cosines of the
// helicity angles and c_k a constant.
#pragma once

#include "fp64_math.cuh"
#include "int_math.cuh"

namespace ipa {

// Constant factors c_k of f_k = c_k f'_k, where f'_k is the product of
// sines and cosines the kernel evaluates (sec. 4 helicity basis).
__device__ const double kBasisScale[10] = {
    1.0, 0.5, 0.5, 1.0, 1.41421356237309504880, -1.41421356237309504880, 1.0 / 3.0,
    0.81649658092772603273, -0.81649658092772603273, 1.15470053837925152902};

// f'_k(cos thK, cos thmu, phi): f_k without its constant factor.
__device__ __forceinline__ void basis_unscaled(double ck, double cl, double phi, const MathTables* mt,
                                               double f[10]) {
    double sp, cp;
    sincos_int(phi, mt, &sp, &cp);
    const double sk2 = fma(-ck, ck, 1.0);
    const double cl2 = cl * cl;
    const double sl2 = 1.0 - cl2;
    const double cp2 = cp * cp;
    const double sksl2 = sk2 * sl2;
    const double q = sqrt(sksl2);                  // sin thK sin thmu
    f[0] = ck * ck * sl2;
    f[1] = sk2 * fma(-sl2, cp2, 1.0);
    f[2] = sk2 * fma(sl2, cp2, cl2);               // sk2 (1 - sl2 sp^2)
    f[3] = sksl2 * (sp * cp);
    const double a = q * (ck * cl);
    f[4] = a * cp;
    f[5] = a * sp;
    f[6] = sl2;
    const double b = q * cl;
    f[7] = b * cp;
    f[8] = b * sp;
    f[9] = ck * sl2;
}

}  // namespace ipa
