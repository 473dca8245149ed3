// Site-local fifth-dimension operators.  Each thread owns one (site, spin *
// colour component, rhs) row of Ls complex numbers, held in registers, so
// every s-coupled operator is a short register recurrence:
//
//   S5 psi_s = P_- psi_{s+1} + P_+ psi_{s-1},  walls -mf      (S5^+ swaps P_+-)
//   L_B      out = scale (b5 + c5 S5) in
//   L_MOOEE  out = scale (d + e S5) in                         (M_ee = M_oo)
//   L_MINV   out = scale (d + e S5)^-1 in
//   L_BMINV  out = scale (b5 + c5 S5)(d + e S5)^-1 in          (commuting factors)
//   L_POST   out = (d + e S5) in + scale (b5 + c5 S5) in2      (tail of M_pc^+)
//            optionally fused with the CG update x += alpha p, r -= alpha out.
//
// Per chirality S5 is a cyclic shift with a -mf twist (S_- on P_+, S_+ on
// P_-, swapped for the adjoint), and (d + e S_-)^-1 has the closed form
// (-a)^k c / (d (1 + mf a^Ls)) (a = -e/d).  It is applied in two sweeps:
// y_0 = [x_0 - mf sum_{t>=1} a^{Ls-t} x_t] / (d (1 + mf a^Ls)), then
// y_s = (x_s - e y_{s-1}) / d; the S_+ case runs the mirror image.
#include "dev_common.cuh"
#include "dwf_internal.cuh"

namespace dwf {

struct LocalArgs {
    int op;
    const void* in;
    const void* in2;
    void* out;
    const int4* tiles;
    int Ls, nrhs, dagger;
    double scale, b5, c5, d, e, mf, a, inv_d, inv_den;
    void* cg_x;
    void* cg_r;
    const void* cg_p;
    const double* alpha;
    const int* run;
    double* partial;
};

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

template <class S, class R, int LSM>
__device__ __forceinline__ void load_row(const S* p, R* xr, R* xi, int Ls) {
#pragma unroll
    for (int s = 0; s < LSM; s += 2)
        if (s < Ls) load_lanes<S, 2, R>(p + 2 * s, xr + s, xi + s);
}

template <class S, class R, int LSM>
__device__ __forceinline__ void store_row(S* p, const R* xr, const R* xi, int Ls) {
#pragma unroll
    for (int s = 0; s < LSM; s += 2)
        if (s < Ls) store_lanes<S, 2, R>(p + 2 * s, xr + s, xi + s);
}

template <class Sin, class Sin2, class Sout, class Svec, class R, int LSM>
__global__ void __launch_bounds__(512) k_local(const LocalArgs a) {
    __shared__ double s_red[512];
    const int4 tl = a.tiles[blockIdx.x];
    const int begin = tl.y, count = tl.z;
    const int Ls = a.Ls, nrhs = a.nrhs;
    const int rows = count * 12 * nrhs;
    const R mf = (R)a.mf, b5 = (R)a.b5, c5 = (R)a.c5, d = (R)a.d, e = (R)a.e;
    const R sc = (R)a.scale;
    double nrm_tot = 0.0;
    // rows are assigned so that one thread always handles the same rhs
    for (int row = threadIdx.x; row < rows; row += blockDim.x) {
        const int r = row % nrhs;
        const int c = (row / nrhs) % 12;
        const int64_t base = ((int64_t)begin * 12 * nrhs + row) * Ls * 2;   // reals
        const bool upper = c < 6;
        // chirality of the shift: non-adjoint P_+ (upper) sees S_-
        const bool down = (upper != (a.dagger != 0));
        R xr[LSM], xi[LSM], yr[LSM], yi[LSM], tr[LSM], ti[LSM];
        load_row<Sin, R, LSM>(reinterpret_cast<const Sin*>(a.in) + base, xr, xi, Ls);
        switch (a.op) {
            case L_B:
            case L_MOOEE: {
                const R c0 = a.op == L_B ? b5 : d;
                const R c1 = a.op == L_B ? c5 : e;
                shift5<R, LSM>(xr, xi, tr, ti, Ls, down, mf);
#pragma unroll
                for (int s = 0; s < LSM; ++s)
                    if (s < Ls) {
                        yr[s] = sc * (c0 * xr[s] + c1 * tr[s]);
                        yi[s] = sc * (c0 * xi[s] + c1 * ti[s]);
                    }
                break;
            }
            case L_MINV:
            case L_BMINV: {
                minv5<R, LSM>(xr, xi, tr, ti, Ls, down, mf, (R)a.a, e, (R)a.inv_d, (R)a.inv_den);
                if (a.op == L_MINV) {
#pragma unroll
                    for (int s = 0; s < LSM; ++s)
                        if (s < Ls) { yr[s] = sc * tr[s]; yi[s] = sc * ti[s]; }
                } else {
                    shift5<R, LSM>(tr, ti, xr, xi, Ls, down, mf);
#pragma unroll
                    for (int s = 0; s < LSM; ++s)
                        if (s < Ls) {
                            yr[s] = sc * (b5 * tr[s] + c5 * xr[s]);
                            yi[s] = sc * (b5 * ti[s] + c5 * xi[s]);
                        }
                }
                break;
            }
            case L_POST: {
                shift5<R, LSM>(xr, xi, tr, ti, Ls, down, mf);
#pragma unroll
                for (int s = 0; s < LSM; ++s)
                    if (s < Ls) { yr[s] = d * xr[s] + e * tr[s]; yi[s] = d * xi[s] + e * ti[s]; }
                load_row<Sin2, R, LSM>(reinterpret_cast<const Sin2*>(a.in2) + base, xr, xi, Ls);
                shift5<R, LSM>(xr, xi, tr, ti, Ls, down, mf);
#pragma unroll
                for (int s = 0; s < LSM; ++s)
                    if (s < Ls) {
                        yr[s] += sc * (b5 * xr[s] + c5 * tr[s]);
                        yi[s] += sc * (b5 * xi[s] + c5 * ti[s]);
                    }
                break;
            }
            default: {   // L_COPY
#pragma unroll
                for (int s = 0; s < LSM; ++s)
                    if (s < Ls) { yr[s] = sc * xr[s]; yi[s] = sc * xi[s]; }
            }
        }
        if (a.cg_r != nullptr) {
            // fused CG step on the vectors: x += alpha p, r -= alpha y, |r|^2
            const int sys = tl.x * nrhs + r;
            const bool run = a.run == nullptr || a.run[sys] != 0;
            const R alpha = (R)a.alpha[sys];
            Svec* rp = reinterpret_cast<Svec*>(a.cg_r) + base;
            load_row<Svec, R, LSM>(rp, tr, ti, Ls);
            if (run) {
                Svec* xp = reinterpret_cast<Svec*>(a.cg_x) + base;
                const Svec* pp = reinterpret_cast<const Svec*>(a.cg_p) + base;
                R pr[LSM], pi[LSM];
                load_row<Svec, R, LSM>(pp, pr, pi, Ls);
                load_row<Svec, R, LSM>(xp, xr, xi, Ls);
#pragma unroll
                for (int s = 0; s < LSM; ++s)
                    if (s < Ls) {
                        xr[s] += alpha * pr[s]; xi[s] += alpha * pi[s];
                        tr[s] -= alpha * yr[s]; ti[s] -= alpha * yi[s];
                    }
                store_row<Svec, R, LSM>(xp, xr, xi, Ls);
                store_row<Svec, R, LSM>(rp, tr, ti, Ls);
            }
            if (a.partial) {
                double nn = 0.0;
#pragma unroll
                for (int s = 0; s < LSM; ++s)
                    if (s < Ls) nn += (double)tr[s] * tr[s] + (double)ti[s] * ti[s];
                nrm_tot += nn;
            }
        } else {
            if (a.out != nullptr)
                store_row<Sout, R, LSM>(reinterpret_cast<Sout*>(a.out) + base, yr, yi, Ls);
            if (a.partial) {
                double nn = 0.0;
#pragma unroll
                for (int s = 0; s < LSM; ++s)
                    if (s < Ls) nn += (double)yr[s] * yr[s] + (double)yi[s] * yi[s];
                nrm_tot += nn;
            }
        }
    }
    if (a.partial) {
        // blockDim.x is a multiple of nrhs, so a thread's rows share one rhs
        const int nr = nrhs;
        block_rhs_reduce(nrm_tot, s_red, nrhs,
                         [&](int t) { return (t < rows) ? t % nr : -1; },
                         a.partial + (size_t)blockIdx.x * nrhs);
    }
}

template <class Sin, class Sin2, class Sout, class Svec, class R>
static dwf_status launch_lt(dwf_handle* h, const LocalCall& c, const TileSet& ts, cudaStream_t s) {
    LocalArgs a;
    const FiveD& f = h->f5[0];
    a.op = c.op;
    a.in = c.in;
    a.in2 = c.in2;
    a.out = c.out;
    a.tiles = ts.d_tiles[c.parity];
    a.Ls = h->p.Ls;
    a.nrhs = c.nrhs;
    a.dagger = c.dagger;
    a.scale = c.scale;
    a.b5 = f.b5; a.c5 = f.c5; a.d = f.d; a.e = f.e; a.mf = f.mf;
    a.a = f.a; a.inv_d = f.inv_d; a.inv_den = f.inv_den;
    a.cg_x = c.cg_x; a.cg_r = c.cg_r; a.cg_p = c.cg_p;
    a.alpha = c.alpha; a.run = c.run; a.partial = c.partial;
    const int nt = ts.ntiles[c.parity];
    if (nt == 0) return DWF_OK;
    // threads: a multiple of nrhs (so every thread keeps one rhs) and of 32
    int l = 32;
    while (l % c.nrhs) l += 32;              // lcm(32, nrhs)
    if (l > 512) {
        set_error("local: lcm(32, nrhs=%d) exceeds 512 threads", c.nrhs);
        return DWF_ERR_UNSUPPORTED;
    }
    const int threads = l * (256 / l > 1 ? 256 / l : 1);
    const int Ls = h->p.Ls;
    if (Ls <= 8)
        k_local<Sin, Sin2, Sout, Svec, R, 8><<<nt, threads, 0, s>>>(a);
    else if (Ls <= 16)
        k_local<Sin, Sin2, Sout, Svec, R, 16><<<nt, threads, 0, s>>>(a);
    else
        k_local<Sin, Sin2, Sout, Svec, R, 32><<<nt, threads, 0, s>>>(a);
    DWF_CUDA(cudaGetLastError());
    return DWF_OK;
}

dwf_status launch_local(dwf_handle* h, const LocalCall& c, cudaStream_t s) {
    const TileSet& ts = get_tiles(h, c.T > 0 ? c.T : 16);
    const dwf_prec pi = c.prec_in, po = c.prec_out;
    const dwf_prec p2 = c.in2 ? c.prec_in2 : pi;
    if (pi == DWF_FP64 || po == DWF_FP64) {
        if (pi != DWF_FP64 || po != DWF_FP64 || p2 != DWF_FP64) return DWF_ERR_UNSUPPORTED;
        return launch_lt<double, double, double, double, double>(h, c, ts, s);
    }
    // FP32 arithmetic; FP32 vectors for the fused CG update
    if (pi == DWF_FP32 && p2 == DWF_FP32 && po == DWF_FP32)
        return launch_lt<float, float, float, float, float>(h, c, ts, s);
    if (pi == DWF_FP32 && p2 == DWF_FP32 && po == DWF_BF16)
        return launch_lt<float, float, bf16, float, float>(h, c, ts, s);
    if (pi == DWF_BF16 && p2 == DWF_BF16 && po == DWF_BF16)
        return launch_lt<bf16, bf16, bf16, float, float>(h, c, ts, s);
    if (pi == DWF_BF16 && p2 == DWF_BF16 && po == DWF_FP32)
        return launch_lt<bf16, bf16, float, float, float>(h, c, ts, s);
    if (pi == DWF_FP32 && p2 == DWF_BF16 && po == DWF_FP32)
        return launch_lt<float, bf16, float, float, float>(h, c, ts, s);
    return DWF_ERR_UNSUPPORTED;
}

}  // namespace dwf
