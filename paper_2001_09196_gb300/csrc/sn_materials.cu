// Materials of one implicit time step of gray thermal radiative transfer in the pseudo-scattering
// form (paper Sec. 4.2, Eq. hohlraum_sigma and Eq. hohlraum_q), one thread per element:
//   b = 16 pi a c T^3,  sigma_t = sigma,  sigma_s = sigma (sigma b) / (C_v/dt + sigma b),
//   q = 4 pi sigma a c T^4 (C_v/dt) / (C_v/dt + sigma b).
// The last line is the printed q_ps = sigma a c T^4 - sigma^2 b a c T^4 / (C_v/dt + sigma b) with the
// two terms combined, so no digits are lost to cancellation when sigma_s is close to sigma; the
// factor 4 pi turns the per-direction source q_ps into the total emission the library's q holds.
#include <cuda_runtime.h>

#include "sn_internal.h"

namespace sn {

namespace {

__global__ void pseudo_scattering_kernel(const double* __restrict__ sigma, const double* __restrict__ cv,
                                         const double* __restrict__ T, int ne, double dt, double a_rad,
                                         double c_light, double* __restrict__ sigma_t, double* __restrict__ sigma_s,
                                         double* __restrict__ q) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const double four_pi = 12.566370614359172953850573533118;
    const double s = sigma[e], t = T[e];
    const double t3 = t * t * t;
    const double sb = s * (4.0 * four_pi * a_rad * c_light * t3);  // sigma b
    const double cdt = cv[e] / dt;
    const double den = cdt + sb;
    sigma_t[e] = s;
    // sigma_ps <= sigma because den >= sigma b; when C_v/dt underflows to 0 the quotient can round
    // one ulp above sigma, so it is capped at sigma (its exact value in that limit)
    sigma_s[e] = fmin(s * sb / den, s);
    q[e] = four_pi * s * a_rad * c_light * t3 * t * cdt / den;
}

}  // namespace

cudaError_t launch_pseudo_scattering(const double* sigma, const double* cv, const double* T, int ne, double dt,
                                     double a_rad, double c_light, double* sigma_t, double* sigma_s, double* q,
                                     cudaStream_t s) {
    if (ne <= 0) return cudaSuccess;
    SN_COUNT_LAUNCH();
    pseudo_scattering_kernel<<<(ne + 255) / 256, 256, 0, s>>>(sigma, cv, T, ne, dt, a_rad, c_light, sigma_t, sigma_s, q);
    return cudaGetLastError();
}

}  // namespace sn
