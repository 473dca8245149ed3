// Fifth-dimension recurrences on one (site, spin-colour, rhs) row of Ls
// complex numbers held in registers (R = float or double; LSM >= Ls is the
// compile-time register extent).  Per chirality S5 is a cyclic shift with a
// -mf twist, and (d + e S_-)^-1 has the closed form a^k / (d (1 + mf a^Ls))
// at shift distance k (a = -e/d), times -mf across the wall.
#pragma once

namespace dwf {

// y = S x for one chirality: down = true is S_- (y_s = x_{s-1}, y_0 = -mf x_{Ls-1}).
template <class R, int LSM>
__device__ __forceinline__ void shift5(const R* xr, const R* xi, R* yr, R* yi, int Ls, bool down,
                                       R mf) {
    if (down) {
        R lr = 0, li = 0;   // x_{Ls-1}, selected with compile-time indices
#pragma unroll
        for (int s = 0; s < LSM; ++s)
            if (s == Ls - 1) { lr = xr[s]; li = xi[s]; }
        yr[0] = -mf * lr;
        yi[0] = -mf * li;
#pragma unroll
        for (int s = 1; s < LSM; ++s)
            if (s < Ls) { yr[s] = xr[s - 1]; yi[s] = xi[s - 1]; }
    } else {
#pragma unroll
        for (int s = 0; s < LSM; ++s) {
            if (s == Ls - 1) { yr[s] = -mf * xr[0]; yi[s] = -mf * xi[0]; }
            else if (s < Ls - 1) {
                yr[s] = xr[s + 1 < LSM ? s + 1 : s];
                yi[s] = xi[s + 1 < LSM ? s + 1 : s];
            }
        }
    }
}

// y = (d + e S)^-1 x for one chirality, S = S_- (down) or S_+.
template <class R, int LSM>
__device__ __forceinline__ void minv5(const R* xr, const R* xi, R* yr, R* yi, int Ls, bool down,
                                      R mf, R a, R e, R inv_d, R inv_den) {
    R accr = 0, acci = 0;
    if (down) {
        // Horner: acc = sum_{t=1}^{Ls-1} a^{Ls-1-t} x_t
#pragma unroll
        for (int t = 1; t < LSM; ++t)
            if (t < Ls) { accr = accr * a + xr[t]; acci = acci * a + xi[t]; }
        yr[0] = (xr[0] - mf * a * accr) * inv_den;
        yi[0] = (xi[0] - mf * a * acci) * inv_den;
#pragma unroll
        for (int s = 1; s < LSM; ++s)
            if (s < Ls) {
                yr[s] = (xr[s] - e * yr[s - 1]) * inv_d;
                yi[s] = (xi[s] - e * yi[s - 1]) * inv_d;
            }
    } else {
        // acc = sum_{t=0}^{Ls-2} a^t x_t
#pragma unroll
        for (int t = LSM - 1; t >= 0; --t)
            if (t <= Ls - 2) { accr = accr * a + xr[t]; acci = acci * a + xi[t]; }
        const int top = Ls - 1;
        R tr = 0, ti = 0;
#pragma unroll
        for (int s = 0; s < LSM; ++s)
            if (s == top) { tr = xr[s]; ti = xi[s]; }
        R yr_top = (tr - mf * a * accr) * inv_den;
        R yi_top = (ti - mf * a * acci) * inv_den;
#pragma unroll
        for (int s = LSM - 1; s >= 0; --s) {
            if (s == top) { yr[s] = yr_top; yi[s] = yi_top; }
            else if (s < top) {
                yr[s] = (xr[s] - e * yr[s + 1 < LSM ? s + 1 : 0]) * inv_d;
                yi[s] = (xi[s] - e * yi[s + 1 < LSM ? s + 1 : 0]) * inv_d;
            }
        }
    }
}

}  // namespace dwf
