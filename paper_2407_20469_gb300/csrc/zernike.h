// zernike.h - Noll-ordered, RMS-normalised Zernike polynomials j = 4..15 in
// Cartesian form, shared by the host plan and the device kernels of this
// library.
//
// The pupil phase phi of Eq. 1 (WSI-APIC, Sec. 2.2) is modelled as
// sum_j c_j Z_j(x, y) at unit-pupil coordinates x = kx / Rx, y = ky / Ry;
// radial orders 2-4 (Noll 4..15) are estimated, piston and tilts (1..3) lie in
// the null space of the difference operator of Eq. 10.
#pragma once

#ifdef __CUDACC__
#define APIC_HD __host__ __device__ __forceinline__
#else
#define APIC_HD inline
#endif

namespace apic {

constexpr int kNumSolved = 12;     // Noll j = 4..15
constexpr int kFirstSolved = 4;

// Writes Z_4..Z_15 at (x, y) into z[0..11]. T is float or double.
template <typename T>
APIC_HD void zernike_4_15(T x, T y, T* z) {
    const T x2 = x * x, y2 = y * y, r2 = x2 + y2, xy = x * y;
    const T s3 = T(1.7320508075688772), s5 = T(2.2360679774997898);
    const T s6 = T(2.4494897427831781), s8 = T(2.8284271247461903);
    const T s10 = T(3.1622776601683795);
    z[0] = s3 * (T(2) * r2 - T(1));                         // Z4  defocus
    z[1] = s6 * T(2) * xy;                                  // Z5  astigmatism, sin 2t
    z[2] = s6 * (x2 - y2);                                  // Z6  astigmatism, cos 2t
    z[3] = s8 * (T(3) * r2 - T(2)) * y;                     // Z7  coma, sin t
    z[4] = s8 * (T(3) * r2 - T(2)) * x;                     // Z8  coma, cos t
    z[5] = s8 * (T(3) * x2 * y - y2 * y);                   // Z9  trefoil, sin 3t
    z[6] = s8 * (x2 * x - T(3) * x * y2);                   // Z10 trefoil, cos 3t
    z[7] = s5 * (T(6) * r2 * r2 - T(6) * r2 + T(1));        // Z11 spherical
    z[8] = s10 * (T(4) * r2 - T(3)) * (x2 - y2);            // Z12 2nd astigmatism, cos 2t
    z[9] = s10 * (T(4) * r2 - T(3)) * T(2) * xy;            // Z13 2nd astigmatism, sin 2t
    z[10] = s10 * (x2 * x2 - T(6) * x2 * y2 + y2 * y2);     // Z14 tetrafoil, cos 4t
    z[11] = s10 * (T(4) * x2 * x * y - T(4) * x * y2 * y);  // Z15 tetrafoil, sin 4t
}

}  // namespace apic
