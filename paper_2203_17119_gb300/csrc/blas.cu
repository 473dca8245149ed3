// Streaming vector kernels of the solvers: precision conversion, per-system
// axpby, and deterministic two-stage FP64 inner products.
//
// A "system" is one (box, rhs) pair: every box of a Dirichlet handle and
// every right-hand side is an independent linear system with its own CG
// scalars.  Stage one writes one FP64 partial per (tile, rhs) in a fixed
// order; stage two sums a box's tiles per rhs with a fixed tree, so results
// are bitwise reproducible run to run.
#include "dev_common.cuh"
#include "dwf_internal.cuh"

namespace dwf {

template <class S>
__device__ __forceinline__ void ld2(const S* p, double& a, double& b) {
    float fr[1], fi[1];
    double dr[1], di[1];
    if constexpr (std::is_same<S, double>::value) {
        load_lanes<S, 1, double>(p, dr, di);
        a = dr[0]; b = di[0];
    } else {
        load_lanes<S, 1, float>(p, fr, fi);
        a = fr[0]; b = fi[0];
    }
}

template <class S>
__device__ __forceinline__ void st2(S* p, double a, double b) {
    if constexpr (std::is_same<S, double>::value) {
        double dr[1] = {a}, di[1] = {b};
        store_lanes<S, 1, double>(p, dr, di);
    } else {
        float fr[1] = {(float)a}, fi[1] = {(float)b};
        store_lanes<S, 1, float>(p, fr, fi);
    }
}

// ---------------------------------------------------------- conversion
template <class Sd, class Ss>
__global__ void k_convert(Sd* __restrict__ dst, const Ss* __restrict__ src, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        double a, b;
        ld2<Ss>(src + 2 * i, a, b);
        st2<Sd>(dst + 2 * i, a, b);
    }
}

template <class Sd>
static dwf_status conv_from(void* dst, const void* src, dwf_prec ps, size_t n, cudaStream_t s) {
    const int threads = 256;
    size_t blocks = (n + threads - 1) / threads;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks == 0) return DWF_OK;
    switch (ps) {
        case DWF_FP64: k_convert<Sd, double><<<blocks, threads, 0, s>>>((Sd*)dst, (const double*)src, n); break;
        case DWF_FP32: k_convert<Sd, float><<<blocks, threads, 0, s>>>((Sd*)dst, (const float*)src, n); break;
        default: k_convert<Sd, bf16><<<blocks, threads, 0, s>>>((Sd*)dst, (const bf16*)src, n); break;
    }
    note_launch();
    DWF_CUDA(cudaGetLastError());
    return DWF_OK;
}

dwf_status launch_convert(void* dst, dwf_prec pd, const void* src, dwf_prec ps, size_t n,
                          cudaStream_t s) {
    switch (pd) {
        case DWF_FP64: return conv_from<double>(dst, src, ps, n, s);
        case DWF_FP32: return conv_from<float>(dst, src, ps, n, s);
        default: return conv_from<bf16>(dst, src, ps, n, s);
    }
}

// ------------------------------------------------------------- axpby
// y = a x + b y on the sites of one parity, a/b per system (array) or fixed.
template <class Sx, class Sy>
__global__ void k_axpby(const int4* __restrict__ tiles, int nrhs, int Ls, const double* a_sys,
                        double a_imm, const Sx* __restrict__ x, const double* b_sys, double b_imm,
                        Sy* __restrict__ y, const int* run) {
    using R = typename std::conditional<std::is_same<Sx, double>::value ||
                                            std::is_same<Sy, double>::value,
                                        double, float>::type;
    const int4 tl = tiles[blockIdx.x];
    const int npair = tl.z * 12 * nrhs * Ls / 2;   // pairs of complex (Ls is even)
    const int64_t off = (int64_t)tl.y * 12 * nrhs * Ls;
    for (int i = threadIdx.x; i < npair; i += blockDim.x) {
        const int r = (2 * i / Ls) % nrhs;
        const int sys = tl.x * nrhs + r;
        if (run != nullptr && run[sys] == 0) continue;
        const R av = (R)(a_sys ? a_sys[sys] : a_imm);
        const R bv = (R)(b_sys ? b_sys[sys] : b_imm);
        R xr[2] = {0, 0}, xi[2] = {0, 0}, yr[2] = {0, 0}, yi[2] = {0, 0};
        if (x != nullptr) load_lanes<Sx, 2, R>(x + 2 * (off + 2 * i), xr, xi);
        if (bv != (R)0) load_lanes<Sy, 2, R>(y + 2 * (off + 2 * i), yr, yi);
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            yr[v] = av * xr[v] + bv * yr[v];
            yi[v] = av * xi[v] + bv * yi[v];
        }
        store_lanes<Sy, 2, R>(y + 2 * (off + 2 * i), yr, yi);
    }
}

template <class Sy>
static dwf_status axpby_y(const int4* tiles, int nt, int nrhs, int Ls, const double* a_sys,
                          double a_imm, const void* x, dwf_prec px, const double* b_sys,
                          double b_imm, void* y, const int* run, cudaStream_t s) {
    if (nt == 0) return DWF_OK;
    switch (px) {
        case DWF_FP64:
            k_axpby<double, Sy><<<nt, 256, 0, s>>>(tiles, nrhs, Ls, a_sys, a_imm, (const double*)x, b_sys, b_imm, (Sy*)y, run);
            break;
        case DWF_FP32:
            k_axpby<float, Sy><<<nt, 256, 0, s>>>(tiles, nrhs, Ls, a_sys, a_imm, (const float*)x, b_sys, b_imm, (Sy*)y, run);
            break;
        default:
            k_axpby<bf16, Sy><<<nt, 256, 0, s>>>(tiles, nrhs, Ls, a_sys, a_imm, (const bf16*)x, b_sys, b_imm, (Sy*)y, run);
    }
    note_launch();
    DWF_CUDA(cudaGetLastError());
    return DWF_OK;
}

dwf_status launch_axpby(dwf_handle* h, int parity, int nrhs, const double* a_sys, double a_imm,
                        const void* x, dwf_prec px, const double* b_sys, double b_imm, void* y,
                        dwf_prec py, const int* run, int T, cudaStream_t s) {
    const TileSet* tsp = nullptr;
    DWF_TRY(get_tiles(h, tile_or_default(T), &tsp));
    const TileSet& ts = *tsp;
    const int nt = ts.ntiles[parity];
    const int4* tl = ts.d_tiles[parity];
    const int Ls = h->p.Ls;
    switch (py) {
        case DWF_FP64: return axpby_y<double>(tl, nt, nrhs, Ls, a_sys, a_imm, x, px, b_sys, b_imm, y, run, s);
        case DWF_FP32: return axpby_y<float>(tl, nt, nrhs, Ls, a_sys, a_imm, x, px, b_sys, b_imm, y, run, s);
        default: return axpby_y<bf16>(tl, nt, nrhs, Ls, a_sys, a_imm, x, px, b_sys, b_imm, y, run, s);
    }
}

// ------------------------------------------------------- inner products
// partial[tile * nrhs + r] = sum over the tile's rows of rhs r of Re <a, b>.
template <class Sa, class Sb>
__global__ void __launch_bounds__(512) k_dot_partial(const int4* __restrict__ tiles, int nrhs,
                                                     int Ls, const Sa* __restrict__ a,
                                                     const Sb* __restrict__ b, double* partial) {
    __shared__ double s_red[512];
    const int4 tl = tiles[blockIdx.x];
    const int rows = tl.z * 12 * nrhs;
    const int64_t off = (int64_t)tl.y * 12 * nrhs * Ls;
    double acc = 0.0;
    // FP64 inputs accumulate in FP64; FP32/BF16 rows sum in FP32, rows in FP64
    using RA = typename std::conditional<std::is_same<Sa, double>::value ||
                                             std::is_same<Sb, double>::value,
                                         double, float>::type;
    for (int row = threadIdx.x; row < rows; row += blockDim.x) {
        const int64_t base = off + (int64_t)row * Ls;
        RA rs = 0;
        for (int s = 0; s < Ls; s += 2) {
            RA ar[2], ai[2], br[2], bi[2];
            load_lanes<Sa, 2, RA>(a + 2 * (base + s), ar, ai);
            if ((const void*)a == (const void*)b) {
                br[0] = ar[0]; bi[0] = ai[0]; br[1] = ar[1]; bi[1] = ai[1];
            } else {
                load_lanes<Sb, 2, RA>(b + 2 * (base + s), br, bi);
            }
            rs += ar[0] * br[0] + ai[0] * bi[0] + ar[1] * br[1] + ai[1] * bi[1];
        }
        acc += (double)rs;
    }
    const int nr = nrhs;
    block_rhs_reduce(acc, s_red, nrhs, [&](int t) { return t < rows ? t % nr : -1; },
                     partial + (size_t)blockIdx.x * nrhs);
}

static int rows_threads(int nrhs) {
    int l = 32;
    while (l % nrhs) l += 32;
    if (l > 512) return -1;
    return l * (256 / l > 1 ? 256 / l : 1);
}

template <class Sa>
static dwf_status dot_a(const int4* tl, int nt, int nrhs, int Ls, const void* a, const void* b,
                        dwf_prec pb, double* partial, cudaStream_t s) {
    const int threads = rows_threads(nrhs);
    if (threads < 0) return DWF_ERR_UNSUPPORTED;
    if (nt == 0) return DWF_OK;
    switch (pb) {
        case DWF_FP64: k_dot_partial<Sa, double><<<nt, threads, 0, s>>>(tl, nrhs, Ls, (const Sa*)a, (const double*)b, partial); break;
        case DWF_FP32: k_dot_partial<Sa, float><<<nt, threads, 0, s>>>(tl, nrhs, Ls, (const Sa*)a, (const float*)b, partial); break;
        default: k_dot_partial<Sa, bf16><<<nt, threads, 0, s>>>(tl, nrhs, Ls, (const Sa*)a, (const bf16*)b, partial);
    }
    note_launch();
    DWF_CUDA(cudaGetLastError());
    return DWF_OK;
}

dwf_status launch_dot_partial(dwf_handle* h, int parity, const void* a, const void* b,
                              dwf_prec pa, dwf_prec pb, int nrhs, double* partial, int T,
                              cudaStream_t s) {
    const TileSet* tsp = nullptr;
    DWF_TRY(get_tiles(h, tile_or_default(T), &tsp));
    const TileSet& ts = *tsp;
    const int nt = ts.ntiles[parity];
    const int4* tl = ts.d_tiles[parity];
    const int Ls = h->p.Ls;
    switch (pa) {
        case DWF_FP64: return dot_a<double>(tl, nt, nrhs, Ls, a, b, pb, partial, s);
        case DWF_FP32: return dot_a<float>(tl, nt, nrhs, Ls, a, b, pb, partial, s);
        default: return dot_a<bf16>(tl, nt, nrhs, Ls, a, b, pb, partial, s);
    }
}

// Stage two: one block per system, fixed-order tree over the box's tiles.
__global__ void k_reduce_sys(const double* __restrict__ partial, const int* __restrict__ box_tb,
                             int nrhs, double* out) {
    __shared__ double s[256];
    const int sys = blockIdx.x;
    const int box = sys / nrhs, r = sys % nrhs;
    const int t0 = box_tb[box], t1 = box_tb[box + 1];
    double acc = 0.0;
    for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) acc += partial[(size_t)t * nrhs + r];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[sys] = s[0];
}

dwf_status launch_reduce_sys(dwf_handle* h, int parity, const double* partial, int nrhs,
                             double* out, int T, cudaStream_t s) {
    const TileSet* ts = nullptr;
    DWF_TRY(get_tiles(h, tile_or_default(T), &ts));
    k_reduce_sys<<<h->nbox * nrhs, 256, 0, s>>>(partial, ts->d_box_tile_begin[parity], nrhs, out);
    note_launch();
    DWF_CUDA(cudaGetLastError());
    return DWF_OK;
}



// ---------------------------------------------------------- copies
// Grid-stride copy of 16-byte vectors with the GPU's own loads and stores, for
// copies between device memory and page-locked host memory: on a CPU-GPU link
// with coherent GPU access to host memory (NVLink-C2C) the SMs' requests keep
// far more bytes in flight than a copy engine.  Streaming cache hints: the data
// is touched once.
__global__ void k_copy16(int4* __restrict__ dst, const int4* __restrict__ src, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        __stcs(dst + i, __ldcs(src + i));
}

// The address the GPU uses for p: device memory as it is, page-locked host
// memory through its device mapping; nullptr for anything else (pageable
// host memory, unknown pointers).
static void* device_view(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();   // clear the error of an unknown pointer
        return nullptr;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return const_cast<void*>(p);
    if (at.type == cudaMemoryTypeHost && at.devicePointer != nullptr) return at.devicePointer;
    return nullptr;
}

dwf_status copy_sm(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    if (dst == nullptr || src == nullptr || bytes % 16 != 0 || ((uintptr_t)dst | (uintptr_t)src) % 16 != 0) {
        set_error("dwf_copy: non-null, 16-byte aligned pointers and a size that is a multiple of 16 bytes");
        return DWF_ERR_ARG;
    }
    if (bytes == 0) return DWF_OK;
    void* d = device_view(dst);
    void* sv = device_view(src);
    if (d == nullptr || sv == nullptr) {
        set_error("dwf_copy: %s is neither device memory nor page-locked host memory", d == nullptr ? "dst" : "src");
        return DWF_ERR_ARG;
    }
    int dev = 0, nsm = 152;
    DWF_CUDA(cudaGetDevice(&dev));
    DWF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const size_t n = bytes / 16;
    size_t blocks = (n + 255) / 256;
    if (blocks > (size_t)nsm * 8) blocks = (size_t)nsm * 8;
    k_copy16<<<(int)blocks, 256, 0, s>>>(static_cast<int4*>(d), static_cast<const int4*>(sv), n);
    note_launch();
    DWF_CUDA(cudaGetLastError());
    return DWF_OK;
}

}  // namespace dwf
