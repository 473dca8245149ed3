// Site-local fifth-dimension operators:
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
// a^k / (d (1 + mf a^Ls)) at shift distance k (a = -e/d), times -mf across
// the wall.
//
// Two designs.  FP64 (k_local): each thread owns one (site, spin * colour,
// rhs) row of Ls numbers in registers and runs the recurrences, so the
// slow FP64 pipe does O(Ls) work per row; (d + e S_-)^-1 takes two sweeps,
// y_0 = [x_0 - mf sum_{t>=1} a^{Ls-t} x_t] / (d (1 + mf a^Ls)), then
// y_s = (x_s - e y_{s-1}) / d, and the S_+ case the mirror image.
// FP32/BF16 (k_local_sparse, k_local_dense): one thread per complex element,
// described below.
#include <algorithm>
#include <map>
#include <utility>
#include <vector>

#include "dev_common.cuh"
#include "dwf_internal.cuh"
#include "fived.cuh"

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

// ---------------------------------------------------------------------
// FP32/BF16 path, one thread per complex element (site, c, rhs, s).
// Persistent blocks walk the tiles; a block stages a chunk of whole rows of
// its tile in shared memory with coalesced, batched loads, then every thread
// forms its own output elements:
//
// * L_B, L_MOOEE, L_POST, L_PB: c0 x_s + c1 (S x)_s, two shared-memory reads.
// * L_MINV, L_BMINV: per chirality the operator is a real Ls x Ls matrix, a
//   polynomial in the twisted shift S (S^Ls = -mf), built once in FP64 on
//   the host.  The row's x_t are read as shared-memory broadcasts (all
//   threads of a row read the same t together), two numbers per 16 bytes.
//
// The block size is a multiple of Ls * nrhs, so a thread's s and rhs never
// change: its matrix rows (both shifts), the s-neighbours, and the CG scalars
// of its system are set up once, and element j of a chunk sits T / Ls rows
// after element j - 1, so no per-element division is needed.  Sums of
// squares are kept in FP32 per chunk and added in FP64 once per chunk.
constexpr int kMatEPT = 4;     // elements per thread per chunk (sparse ops)
constexpr int kDenseEPT = 4;   // (dense ops: fewer, their matrix rows take the registers)

struct LocalMatArgs {
    int op;
    const void* in;
    const void* in2;
    void* out;
    const int4* tiles;
    int ntiles;
    int Ls, LsP, nrhs, dagger;     // LsP: Ls rounded up to even (shared row stride)
    float scale, b5, c5, d, e, mf;
    const float* mats;             // [4 ops][2 shifts][Ls][Ls]
    void* cg_x;
    void* cg_r;
    const void* cg_p;
    const double* alpha;
    const int* run;
    double* partial;
};

// Per-tile |.|^2 sums: thread t's elements all belong to rhs (t / Ls) % nrhs.
__device__ __forceinline__ void mat_partial(const LocalMatArgs& a, double nrm, double* s_red, int tile) {
    const int nr = a.nrhs, L = a.Ls;
    block_rhs_reduce(nrm, s_red, nr, [&](int t) { return (t / L) % nr; },
                     a.partial + (size_t)tile * nr);
}

template <class Sin, class Sin2, class Sout, class Svec, bool FIXC>
__global__ void __launch_bounds__(FIXC ? 512 : 256, FIXC ? 2 : 4) k_local_sparse(const LocalMatArgs a) {
    extern __shared__ __align__(16) float smem_f[];
    __shared__ double s_red[512];
    const int Ls = a.Ls, LsP = a.LsP, nrhs = a.nrhs, N5 = Ls * nrhs, T = blockDim.x;
    const int tid = threadIdx.x;
    const int s = tid % Ls, row0 = tid / Ls, drow = T / Ls;
    const int rhs = row0 % nrhs;
    const int cq0 = tid / N5, dcq = T / N5;
    const int chunk = T * kMatEPT;
    float2* xs = reinterpret_cast<float2*>(smem_f);
    float2* x2 = xs + (size_t)(chunk / Ls) * LsP;
    const int op = a.op;
    const bool two = op == L_POST, pb = op == L_PB, cg = a.cg_r != nullptr;
    const bool part = a.partial != nullptr;
    const float c0 = (op == L_MOOEE || op == L_POST) ? a.d : a.b5;
    const float c1 = (op == L_MOOEE || op == L_POST) ? a.e : a.c5;
    // s-neighbours: S_- reads s - 1 (wall: -mf x_{Ls-1}), S_+ reads s + 1
    const int nb_dn = s > 0 ? s - 1 : Ls - 1, nb_up = s < Ls - 1 ? s + 1 : 0;
    const float tw_dn = s > 0 ? 1.f : -a.mf, tw_up = s < Ls - 1 ? 1.f : -a.mf;
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const int4 tl = a.tiles[tile];
        const int nel = tl.z * 12 * N5;
        const int64_t base = (int64_t)tl.y * 12 * N5;
        float coef = 0.f;
        bool live = true;
        if (pb || cg) {
            const int sys = tl.x * nrhs + rhs;
            coef = (float)a.alpha[sys];
            live = a.run == nullptr || a.run[sys] != 0;
        }
        double nrm = 0.0;
        for (int ch = 0; ch < nel; ch += chunk) {
            const int n = min(chunk, nel - ch);
            const int64_t g0 = base + ch + tid;
            const int cq = ch / N5 + cq0;
            __syncthreads();   // the previous chunk is no longer read
            float2 v[kMatEPT], w[kMatEPT];
#pragma unroll
            for (int j = 0; j < kMatEPT; ++j) {
                if (tid + j * T < n) {
                    const int64_t g = g0 + (int64_t)j * T;
                    float xr[1], xi[1];
                    if (pb) load_lanes<Svec, 1, float>(reinterpret_cast<const Svec*>(a.cg_p) + 2 * g, xr, xi);
                    else load_lanes<Sin, 1, float>(reinterpret_cast<const Sin*>(a.in) + 2 * g, xr, xi);
                    v[j] = make_float2(xr[0], xi[0]);
                    if (pb || two) {   // L_PB: r;  L_POST: the B operand
                        load_lanes<Sin2, 1, float>(reinterpret_cast<const Sin2*>(a.in2) + 2 * g, xr, xi);
                        w[j] = make_float2(xr[0], xi[0]);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < kMatEPT; ++j) {
                if (tid + j * T < n) {
                    float2 x = v[j];
                    if (pb && live) {   // p = r + beta p
                        x = make_float2(fmaf(coef, x.x, w[j].x), fmaf(coef, x.y, w[j].y));
                        float pr[1] = {x.x}, pi[1] = {x.y};
                        store_lanes<Svec, 1, float>(
                            reinterpret_cast<Svec*>(const_cast<void*>(a.cg_p)) + 2 * (g0 + (int64_t)j * T), pr, pi);
                    }
                    const int k = (row0 + j * drow) * LsP + s;
                    xs[k] = x;
                    if (two) x2[k] = w[j];
                }
            }
            __syncthreads();
            float pn = 0.f;
#pragma unroll
            for (int j = 0; j < kMatEPT; ++j) {
                if (tid + j * T >= n) continue;
                const int row = row0 + j * drow;
                const int c = FIXC ? cq0 % 12 : (cq + j * dcq) % 12;   // FIXC: fixed per thread
                const bool down = (c < 6) != (a.dagger != 0);   // S_- (else S_+)
                const int nb = down ? nb_dn : nb_up;
                const float tw = down ? tw_dn : tw_up;
                const float2 xv = xs[row * LsP + s], xn = xs[row * LsP + nb];
                float yr = fmaf(c1 * tw, xn.x, c0 * xv.x), yi = fmaf(c1 * tw, xn.y, c0 * xv.y);
                if (two) {
                    const float2 zv = x2[row * LsP + s], zn = x2[row * LsP + nb];
                    const float zr = fmaf(a.c5 * tw, zn.x, a.b5 * zv.x);
                    const float zi = fmaf(a.c5 * tw, zn.y, a.b5 * zv.y);
                    yr = fmaf(a.scale, zr, yr);
                    yi = fmaf(a.scale, zi, yi);
                } else {
                    yr *= a.scale;
                    yi *= a.scale;
                }
                const int64_t g = g0 + (int64_t)j * T;
                if (cg) {   // fused CG update: x += alpha p, r -= alpha y
                    Svec* rp = reinterpret_cast<Svec*>(a.cg_r) + 2 * g;
                    float rr[1], ri[1];
                    load_lanes<Svec, 1, float>(rp, rr, ri);
                    if (live) {
                        Svec* xp = reinterpret_cast<Svec*>(a.cg_x) + 2 * g;
                        float xr[1], xi[1], pr[1], pi[1];
                        load_lanes<Svec, 1, float>(xp, xr, xi);
                        load_lanes<Svec, 1, float>(reinterpret_cast<const Svec*>(a.cg_p) + 2 * g, pr, pi);
                        xr[0] = fmaf(coef, pr[0], xr[0]);
                        xi[0] = fmaf(coef, pi[0], xi[0]);
                        rr[0] = fmaf(-coef, yr, rr[0]);
                        ri[0] = fmaf(-coef, yi, ri[0]);
                        store_lanes<Svec, 1, float>(xp, xr, xi);
                        store_lanes<Svec, 1, float>(rp, rr, ri);
                    }
                    pn = fmaf(rr[0], rr[0], fmaf(ri[0], ri[0], pn));
                } else {
                    float orr[1] = {yr}, oi[1] = {yi};
                    if (a.out != nullptr) store_lanes<Sout, 1, float, true>(reinterpret_cast<Sout*>(a.out) + 2 * g, orr, oi);
                    pn = fmaf(yr, yr, fmaf(yi, yi, pn));
                }
            }
            if (part) nrm += (double)pn;
        }
        if (part) mat_partial(a, nrm, s_red, tile);
    }
}

// FIXC: the block size is a multiple of 12 Ls nrhs, so a thread's spin-colour
// row c, hence its chirality, is fixed too and it keeps one matrix row.
template <class Sin, class Sout, int LSM, bool FIXC>
__global__ void __launch_bounds__(FIXC ? 512 : 256, FIXC ? 2 : (LSM <= 16 ? 3 : 2))
    k_local_dense(const LocalMatArgs a) {
    extern __shared__ __align__(16) float smem_f[];
    __shared__ double s_red[512];
    const int Ls = a.Ls, LsP = a.LsP, nrhs = a.nrhs, N5 = Ls * nrhs, T = blockDim.x;
    const int tid = threadIdx.x;
    const int s = tid % Ls, row0 = tid / Ls, drow = T / Ls;
    const int cq0 = tid / N5, dcq = T / N5;
    const int chunk = T * kDenseEPT;
    float2* xs = reinterpret_cast<float2*>(smem_f);
    const bool part = a.partial != nullptr;
    const int m = a.op == L_MINV ? 2 : 3;
    // this thread's matrix rows, S_- and S_+ (FIXC: only its chirality's), scale folded in
    constexpr int NROW = FIXC ? 1 : 2;
    float cf[NROW][LSM];
    const bool down0 = ((cq0 % 12) < 6) != (a.dagger != 0);   // FIXC: the thread's shift
#pragma unroll
    for (int q = 0; q < NROW; ++q) {
        const int sh = FIXC ? (down0 ? 0 : 1) : q;
#pragma unroll
        for (int t = 0; t < LSM; ++t)
            cf[q][t] = t < Ls ? a.scale * a.mats[((size_t)m * 2 + sh) * Ls * Ls + s * Ls + t] : 0.f;
    }
    for (int r = tid; r < chunk / Ls; r += T)   // pad column read by the paired loads
        if (LsP != Ls) xs[r * LsP + Ls] = make_float2(0.f, 0.f);
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const int4 tl = a.tiles[tile];
        const int nel = tl.z * 12 * N5;
        const int64_t base = (int64_t)tl.y * 12 * N5;
        double nrm = 0.0;
        for (int ch = 0; ch < nel; ch += chunk) {
            const int n = min(chunk, nel - ch);
            const int64_t g0 = base + ch + tid;
            const int cq = ch / N5 + cq0;
            __syncthreads();
            float2 v[kDenseEPT];
#pragma unroll
            for (int j = 0; j < kDenseEPT; ++j) {
                if (tid + j * T < n) {
                    float xr[1], xi[1];
                    load_lanes<Sin, 1, float>(reinterpret_cast<const Sin*>(a.in) + 2 * (g0 + (int64_t)j * T), xr, xi);
                    v[j] = make_float2(xr[0], xi[0]);
                }
            }
#pragma unroll
            for (int j = 0; j < kDenseEPT; ++j)
                if (tid + j * T < n) xs[(row0 + j * drow) * LsP + s] = v[j];
            __syncthreads();
            float pn = 0.f;
#pragma unroll
            for (int j = 0; j < kDenseEPT; ++j) {
                if (tid + j * T >= n) continue;
                const float4* xrow = reinterpret_cast<const float4*>(xs + (row0 + j * drow) * LsP);
                float yr = 0.f, yi = 0.f;
                const bool down = FIXC ? true : (((cq + j * dcq) % 12) < 6) != (a.dagger != 0);
                const int q0 = FIXC ? 0 : (down ? 0 : 1);
                if (FIXC || q0 == 0) {
#pragma unroll
                    for (int t = 0; t < LSM; t += 2)
                        if (t < Ls) {
                            const float4 q = xrow[t / 2];
                            yr = fmaf(cf[0][t], q.x, yr); yi = fmaf(cf[0][t], q.y, yi);
                            yr = fmaf(cf[0][t + 1], q.z, yr); yi = fmaf(cf[0][t + 1], q.w, yi);
                        }
                } else {
#pragma unroll
                    for (int t = 0; t < LSM; t += 2)
                        if (t < Ls) {
                            const float4 q = xrow[t / 2];
                            yr = fmaf(cf[NROW - 1][t], q.x, yr); yi = fmaf(cf[NROW - 1][t], q.y, yi);
                            yr = fmaf(cf[NROW - 1][t + 1], q.z, yr); yi = fmaf(cf[NROW - 1][t + 1], q.w, yi);
                        }
                }
                float orr[1] = {yr}, oi[1] = {yi};
                if (a.out != nullptr)
                    store_lanes<Sout, 1, float, true>(reinterpret_cast<Sout*>(a.out) + 2 * (g0 + (int64_t)j * T), orr, oi);
                pn = fmaf(yr, yr, fmaf(yi, yi, pn));
            }
            if (part) nrm += (double)pn;
        }
        if (part) mat_partial(a, nrm, s_red, tile);
    }
}

// Host-side matrices of the fifth-dimension operators, FP64 -> FP32:
// [op][shift][s][t], op 0: b5 + c5 S, 1: d + e S, 2: (d + e S)^-1,
// 3: (b5 + c5 S)(d + e S)^-1; shift 0: S_-, 1: S_+.
void build_fived_mats(const FiveD& f, std::vector<float>& out) {
    const int L = f.Ls;
    out.assign((size_t)8 * L * L, 0.f);
    for (int sh = 0; sh < 2; ++sh) {
        // S_-: y_s = x_{s-1}, y_0 = -mf x_{L-1};  S_+: y_s = x_{s+1}, y_{L-1} = -mf x_0
        std::vector<double> S((size_t)L * L, 0.0);
        for (int s = 0; s < L; ++s) {
            if (sh == 0) S[s * L + (s == 0 ? L - 1 : s - 1)] = s == 0 ? -f.mf : 1.0;
            else S[s * L + (s == L - 1 ? 0 : s + 1)] = s == L - 1 ? -f.mf : 1.0;
        }
        std::vector<double> B((size_t)L * L), M((size_t)L * L), Mi((size_t)L * L, 0.0), BMi((size_t)L * L, 0.0);
        for (int i = 0; i < L * L; ++i) {
            const double id = (i / L == i % L) ? 1.0 : 0.0;
            B[i] = f.b5 * id + f.c5 * S[i];
            M[i] = f.d * id + f.e * S[i];
        }
        // (d + e S)^-1 = sum_k a^k S^k / (d (1 + mf a^L)), a = -e/d: entry (s, t)
        // is a^k inv_den with k the shift distance, times -mf across the wall.
        for (int s = 0; s < L; ++s)
            for (int t = 0; t < L; ++t) {
                const int k = sh == 0 ? ((s - t) % L + L) % L : ((t - s) % L + L) % L;
                const bool wrap = sh == 0 ? (t > s) : (t < s);
                double v = f.inv_den;
                for (int q = 0; q < k; ++q) v *= f.a;
                Mi[s * L + t] = wrap ? -f.mf * v : v;
            }
        for (int s = 0; s < L; ++s)
            for (int t = 0; t < L; ++t) {
                double acc = 0.0;
                for (int q = 0; q < L; ++q) acc += B[s * L + q] * Mi[q * L + t];
                BMi[s * L + t] = acc;
            }
        const std::vector<double>* ops[4] = {&B, &M, &Mi, &BMi};
        for (int o = 0; o < 4; ++o)
            for (int i = 0; i < L * L; ++i) out[((size_t)o * 2 + sh) * L * L + i] = (float)(*ops[o])[i];
    }
}

template <class K>
static cudaError_t mat_attr(K kern) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
}

dwf_status init_local_mat_kernels() {
#define DWF_SPARSE_ATTR(A, B, C, D)                         \
    DWF_CUDA(mat_attr(k_local_sparse<A, B, C, D, false>));  \
    DWF_CUDA(mat_attr(k_local_sparse<A, B, C, D, true>));
    DWF_SPARSE_ATTR(float, float, float, float)
    DWF_SPARSE_ATTR(float, float, bf16, float)
    DWF_SPARSE_ATTR(bf16, bf16, bf16, float)
    DWF_SPARSE_ATTR(bf16, bf16, float, float)
    DWF_SPARSE_ATTR(float, bf16, float, float)
#undef DWF_SPARSE_ATTR
#define DWF_DENSE_ATTR(A, B)                                                     \
    DWF_CUDA(mat_attr(k_local_dense<A, B, 12, false>));                          \
    DWF_CUDA(mat_attr(k_local_dense<A, B, 16, false>));                          \
    DWF_CUDA(mat_attr(k_local_dense<A, B, 32, false>));                          \
    DWF_CUDA(mat_attr(k_local_dense<A, B, 12, true>));                           \
    DWF_CUDA(mat_attr(k_local_dense<A, B, 16, true>));                           \
    DWF_CUDA(mat_attr(k_local_dense<A, B, 32, true>));
    DWF_DENSE_ATTR(float, float)
    DWF_DENSE_ATTR(float, bf16)
    DWF_DENSE_ATTR(bf16, bf16)
    DWF_DENSE_ATTR(bf16, float)
#undef DWF_DENSE_ATTR
    return DWF_OK;
}

// Block size: a multiple of lcm(32, 12 Ls nrhs) up to 512 when one exists
// (*fixc: every thread keeps one spin-colour row and chirality), else the
// largest multiple of lcm(32, Ls nrhs) up to 256, or -1 (then the rows
// kernel serves).
static int lcm32(int n, int cap) {
    int l = 32;
    while (l % n && l <= cap) l += 32;
    return l <= cap ? l : -1;
}

static int mat_threads(int N5, bool* fixc = nullptr) {
    const int l12 = lcm32(12 * N5, 512);
    if (l12 > 0) {
        if (fixc) *fixc = true;
        return l12 * std::max(1, 256 / l12);
    }
    if (fixc) *fixc = false;
    const int l = lcm32(N5, 256);
    return l > 0 ? l * (256 / l) : -1;
}

static LocalMatArgs mat_args(dwf_handle* h, const LocalCall& c, const TileSet& ts) {
    const FiveD& f = h->f5[0];
    LocalMatArgs a;
    a.op = c.op;
    a.in = c.in;
    a.in2 = c.in2;
    a.out = c.out;
    a.tiles = ts.d_tiles[c.parity];
    a.ntiles = ts.ntiles[c.parity];
    a.Ls = f.Ls;
    a.LsP = f.Ls + (f.Ls & 1);
    a.nrhs = c.nrhs;
    a.dagger = c.dagger;
    a.scale = (float)c.scale;
    a.b5 = (float)f.b5; a.c5 = (float)f.c5; a.d = (float)f.d; a.e = (float)f.e; a.mf = (float)f.mf;
    a.mats = h->d_mats;
    a.cg_x = c.cg_x; a.cg_r = c.cg_r; a.cg_p = c.cg_p;
    a.alpha = c.alpha; a.run = c.run; a.partial = c.partial;
    return a;
}


template <class Sin, class Sin2, class Sout, class Svec>
static dwf_status launch_mat(dwf_handle* h, const LocalCall& c, const TileSet& ts, cudaStream_t s) {
    const int nt = ts.ntiles[c.parity];
    if (nt == 0) return DWF_OK;
    const int Ls = h->p.Ls;
    bool fixc = false;
    const int T = mat_threads(Ls * c.nrhs, &fixc);
    const LocalMatArgs a = mat_args(h, c, ts);
    void (*kern)(const LocalMatArgs);
    size_t smem;
    if (c.op == L_MINV || c.op == L_BMINV) {
        smem = (size_t)T * kDenseEPT / Ls * a.LsP * sizeof(float2);
        if (fixc)
            kern = Ls <= 12 ? k_local_dense<Sin, Sout, 12, true>
                 : Ls <= 16 ? k_local_dense<Sin, Sout, 16, true> : k_local_dense<Sin, Sout, 32, true>;
        else
            kern = Ls <= 12 ? k_local_dense<Sin, Sout, 12, false>
                 : Ls <= 16 ? k_local_dense<Sin, Sout, 16, false> : k_local_dense<Sin, Sout, 32, false>;
    } else {
        smem = (size_t)(c.op == L_POST ? 2 : 1) * T * kMatEPT / Ls * a.LsP * sizeof(float2);
        kern = fixc ? k_local_sparse<Sin, Sin2, Sout, Svec, true> : k_local_sparse<Sin, Sin2, Sout, Svec, false>;
    }
    int grid = 0;
    dwf_status st = persistent_grid((const void*)kern, T, smem, nt, &grid);
    if (st != DWF_OK) return st;
    kern<<<grid, T, smem, s>>>(a);
    note_launch();
    DWF_CUDA(cudaGetLastError());
    return DWF_OK;
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
    const FiveD& f = c.f5 ? *c.f5 : h->f5[0];
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
    const TileSet* tsp = nullptr;
    DWF_TRY(get_tiles(h, tile_or_default(c.T), &tsp));
    const TileSet& ts = *tsp;
    const dwf_prec pi = c.prec_in, po = c.prec_out;
    const dwf_prec p2 = c.in2 ? c.prec_in2 : pi;
    if (c.f5 != nullptr && (pi != DWF_FP64 || po != DWF_FP64)) return DWF_ERR_UNSUPPORTED;
    if (pi == DWF_FP64 || po == DWF_FP64) {
        if (pi != DWF_FP64 || po != DWF_FP64 || p2 != DWF_FP64) return DWF_ERR_UNSUPPORTED;
        return launch_lt<double, double, double, double, double>(h, c, ts, s);
    }
    // FP32 arithmetic; FP32 vectors for the fused CG updates.  The matrix
    // kernel when Ls * nrhs allows a fixed rhs per thread, else the rows kernel.
    const bool dense_op = c.op == L_MINV || c.op == L_BMINV;
    if (c.op != L_COPY && !(dense_op && c.cg_r != nullptr) && mat_threads(h->p.Ls * c.nrhs) > 0 &&
        h->d_mats != nullptr) {
        if (pi == DWF_FP32 && p2 == DWF_FP32 && po == DWF_FP32)
            return launch_mat<float, float, float, float>(h, c, ts, s);
        if (pi == DWF_FP32 && p2 == DWF_FP32 && po == DWF_BF16)
            return launch_mat<float, float, bf16, float>(h, c, ts, s);
        if (pi == DWF_BF16 && p2 == DWF_BF16 && po == DWF_BF16)
            return launch_mat<bf16, bf16, bf16, float>(h, c, ts, s);
        if (pi == DWF_BF16 && p2 == DWF_BF16 && po == DWF_FP32)
            return launch_mat<bf16, bf16, float, float>(h, c, ts, s);
        if (pi == DWF_FP32 && p2 == DWF_BF16 && po == DWF_FP32)
            return launch_mat<float, bf16, float, float>(h, c, ts, s);
    }
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
