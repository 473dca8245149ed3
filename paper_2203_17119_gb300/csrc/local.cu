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
//   L_PB     p = r + beta p (CG direction update), out = scale (b5 + c5 S5) p
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

// One pass over a tile, in blocks of RB = blockDim rows:
//   1. coalesced vector loads of the block's rows (and of a second input)
//      into shared memory, planes re/im with row stride Ls + 1;
//   2. one thread per row applies the s-coupled operator in registers and
//      writes the row back;
//   3. coalesced epilogue: store, or the fused CG update of the vectors;
//   4. per-row |.|^2 for the deterministic per-(tile, rhs) partial sums.
// L_PB (the CG direction update fused with the next pre-op) does
// p = r + beta p in step 1 (p: cg_p, read and written; r: in2; beta: alpha
// array) and out = scale (b5 + c5 S5) p in step 2.
template <class Sin, class Sin2, class Sout, class Svec, class R, int LSM>
__global__ void __launch_bounds__(512) k_local(const LocalArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double s_red[512];
    const int Ls = a.Ls, nrhs = a.nrhs;
    const int RB = blockDim.x;
    const int stride = Ls + 1;
    R* Are = reinterpret_cast<R*>(smem_raw);
    R* Aim = Are + RB * stride;
    R* Bre = Aim + RB * stride;
    R* Bim = Bre + RB * stride;
    const int4 tl = a.tiles[blockIdx.x];
    const int rows_total = tl.z * 12 * nrhs;
    const int64_t tile_base = (int64_t)tl.y * 12 * nrhs * Ls;   // complex offset
    const bool two = a.op == L_POST;
    const bool cg = a.cg_r != nullptr;
    const bool pb = a.op == L_PB;
    const R mf = (R)a.mf, b5 = (R)a.b5, c5 = (R)a.c5, d = (R)a.d, e = (R)a.e;
    const R sc = (R)a.scale;
    double nrm = 0.0;
    for (int rb0 = 0; rb0 < rows_total; rb0 += RB) {
        const int nrows = min(RB, rows_total - rb0);
        const int npair = nrows * Ls / 2;
        const int64_t base = tile_base + (int64_t)rb0 * Ls;
        // 1. loads
        for (int i = threadIdx.x; i < npair; i += blockDim.x) {
            const int c0 = 2 * i;
            const int row = c0 / Ls, s = c0 - row * Ls;
            R xr[2], xi[2];
            if (pb) {
                const int sys = tl.x * nrhs + (rb0 + row) % nrhs;
                Svec* pp = reinterpret_cast<Svec*>(const_cast<void*>(a.cg_p)) + 2 * (base + c0);
                load_lanes<Svec, 2, R>(pp, xr, xi);
                if (a.run == nullptr || a.run[sys] != 0) {
                    R rr[2], ri[2];   // r is the second input of L_PB
                    load_lanes<Sin2, 2, R>(reinterpret_cast<const Sin2*>(a.in2) + 2 * (base + c0), rr, ri);
                    const R beta = (R)a.alpha[sys];
                    xr[0] = rr[0] + beta * xr[0]; xi[0] = ri[0] + beta * xi[0];
                    xr[1] = rr[1] + beta * xr[1]; xi[1] = ri[1] + beta * xi[1];
                    store_lanes<Svec, 2, R>(pp, xr, xi);
                }
            } else {
                load_lanes<Sin, 2, R>(reinterpret_cast<const Sin*>(a.in) + 2 * (base + c0), xr, xi);
            }
            Are[row * stride + s] = xr[0]; Are[row * stride + s + 1] = xr[1];
            Aim[row * stride + s] = xi[0]; Aim[row * stride + s + 1] = xi[1];
            if (two) {
                load_lanes<Sin2, 2, R>(reinterpret_cast<const Sin2*>(a.in2) + 2 * (base + c0), xr, xi);
                Bre[row * stride + s] = xr[0]; Bre[row * stride + s + 1] = xr[1];
                Bim[row * stride + s] = xi[0]; Bim[row * stride + s + 1] = xi[1];
            }
        }
        __syncthreads();
        // 2. one row per thread
        if ((int)threadIdx.x < nrows) {
            const int row = threadIdx.x;
            const int c = ((rb0 + row) / nrhs) % 12;
            // chirality of the shift: non-adjoint P_+ (upper spins) sees S_-
            const bool down = ((c < 6) != (a.dagger != 0));
            R xr[LSM], xi[LSM], yr[LSM], yi[LSM], tr[LSM], ti[LSM];
#pragma unroll
            for (int s = 0; s < LSM; ++s)
                if (s < Ls) { xr[s] = Are[row * stride + s]; xi[s] = Aim[row * stride + s]; }
            switch (a.op) {
                case L_B:
                case L_PB:
                case L_MOOEE: {
                    const R c0 = a.op == L_MOOEE ? d : b5;
                    const R c1 = a.op == L_MOOEE ? e : c5;
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
#pragma unroll
                    for (int s = 0; s < LSM; ++s)
                        if (s < Ls) { xr[s] = Bre[row * stride + s]; xi[s] = Bim[row * stride + s]; }
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
#pragma unroll
            for (int s = 0; s < LSM; ++s)
                if (s < Ls) { Are[row * stride + s] = yr[s]; Aim[row * stride + s] = yi[s]; }
        }
        __syncthreads();
        // 3. epilogue
        for (int i = threadIdx.x; i < npair; i += blockDim.x) {
            const int c0 = 2 * i;
            const int row = c0 / Ls, s = c0 - row * Ls;
            R yr[2] = {Are[row * stride + s], Are[row * stride + s + 1]};
            R yi[2] = {Aim[row * stride + s], Aim[row * stride + s + 1]};
            if (cg) {
                const int sys = tl.x * nrhs + (rb0 + row) % nrhs;
                Svec* rp = reinterpret_cast<Svec*>(a.cg_r) + 2 * (base + c0);
                R rr[2], ri[2];
                load_lanes<Svec, 2, R>(rp, rr, ri);
                if (a.run == nullptr || a.run[sys] != 0) {
                    const R alpha = (R)a.alpha[sys];
                    Svec* xp = reinterpret_cast<Svec*>(a.cg_x) + 2 * (base + c0);
                    R xr[2], xi[2], pr[2], pi[2];
                    load_lanes<Svec, 2, R>(xp, xr, xi);
                    load_lanes<Svec, 2, R>(reinterpret_cast<const Svec*>(a.cg_p) + 2 * (base + c0), pr, pi);
#pragma unroll
                    for (int v = 0; v < 2; ++v) {
                        xr[v] += alpha * pr[v]; xi[v] += alpha * pi[v];
                        rr[v] -= alpha * yr[v]; ri[v] -= alpha * yi[v];
                    }
                    store_lanes<Svec, 2, R>(xp, xr, xi);
                    store_lanes<Svec, 2, R>(rp, rr, ri);
                }
                Bre[row * stride + s] = rr[0]; Bre[row * stride + s + 1] = rr[1];
                Bim[row * stride + s] = ri[0]; Bim[row * stride + s + 1] = ri[1];
            } else if (a.out != nullptr) {
                store_lanes<Sout, 2, R>(reinterpret_cast<Sout*>(a.out) + 2 * (base + c0), yr, yi);
            }
        }
        if (a.partial) {
            __syncthreads();
            // 4. per-row |.|^2 (of the updated residual for the CG step)
            if ((int)threadIdx.x < nrows) {
                const R* pr = cg ? Bre : Are;
                const R* pi = cg ? Bim : Aim;
                R acc = 0;
                for (int s = 0; s < Ls; ++s) {
                    const R u = pr[threadIdx.x * stride + s], v = pi[threadIdx.x * stride + s];
                    acc += u * u + v * v;
                }
                nrm += (double)acc;
            }
        }
        __syncthreads();
    }
    if (a.partial) {
        // blockDim.x is a multiple of nrhs: thread t's rows all have rhs t % nrhs
        const int nr = nrhs;
        block_rhs_reduce(nrm, s_red, nrhs, [&](int t) { return t % nr; },
                         a.partial + (size_t)blockIdx.x * nrhs);
    }
}

template <class R>
static int local_threads(int nrhs) {
    int l = 32;
    while (l % nrhs) l += 32;                  // lcm(32, nrhs)
    if (l > 512) return -1;
    const int target = sizeof(R) == 8 ? 128 : 256;
    return l >= target ? l : l * (target / l);
}

template <class R>
static size_t local_smem(int threads, int Ls) {
    return (size_t)4 * threads * (Ls + 1) * sizeof(R);
}

template <class Sin, class Sin2, class Sout, class Svec, class R, int LSM>
static cudaError_t local_attr() {
    return cudaFuncSetAttribute(k_local<Sin, Sin2, Sout, Svec, R, LSM>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

template <class Sin, class Sin2, class Sout, class Svec, class R>
static cudaError_t local_attr_all() {
    cudaError_t e1 = local_attr<Sin, Sin2, Sout, Svec, R, 8>();
    cudaError_t e2 = local_attr<Sin, Sin2, Sout, Svec, R, 16>();
    cudaError_t e3 = local_attr<Sin, Sin2, Sout, Svec, R, 32>();
    return e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3);
}

dwf_status init_local_kernels() {
    DWF_CUDA((local_attr_all<double, double, double, double, double>()));
    DWF_CUDA((local_attr_all<float, float, float, float, float>()));
    DWF_CUDA((local_attr_all<float, float, bf16, float, float>()));
    DWF_CUDA((local_attr_all<bf16, bf16, bf16, float, float>()));
    DWF_CUDA((local_attr_all<bf16, bf16, float, float, float>()));
    DWF_CUDA((local_attr_all<float, bf16, float, float, float>()));
    return DWF_OK;
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
    const int threads = local_threads<R>(c.nrhs);
    if (threads < 0) {
        set_error("local: lcm(32, nrhs=%d) exceeds 512 threads", c.nrhs);
        return DWF_ERR_UNSUPPORTED;
    }
    const int Ls = h->p.Ls;
    const size_t smem = local_smem<R>(threads, Ls);
    if (smem > 200 * 1024) {
        set_error("local: %zu bytes of shared memory for nrhs=%d, Ls=%d", smem, c.nrhs, Ls);
        return DWF_ERR_UNSUPPORTED;
    }
    if (Ls <= 8)
        k_local<Sin, Sin2, Sout, Svec, R, 8><<<nt, threads, smem, s>>>(a);
    else if (Ls <= 16)
        k_local<Sin, Sin2, Sout, Svec, R, 16><<<nt, threads, smem, s>>>(a);
    else
        k_local<Sin, Sin2, Sout, Svec, R, 32><<<nt, threads, smem, s>>>(a);
    note_launch();
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
    // FP32 arithmetic; FP32 vectors for the fused CG updates
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
