// Device helpers: typed loads/stores of consecutive complex lanes, BF16
// conversion, bulk-copy (TMA) + mbarrier wrappers with bounded waits.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>
#include <type_traits>

namespace dwf {

using bf16 = __nv_bfloat16;

// Number of try_wait polls before a wait is declared lost (each poll blocks
// for a bounded, hardware-defined time slice: well under a second in total).
constexpr int kWaitPolls = 1 << 20;

// device error word bits
constexpr int kErrBulkTimeout = 1;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// 1D bulk copy global -> shared, completion counted on `bar` (bytes % 16 == 0,
// both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bounded wait; returns false if the phase did not complete in time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase) {
    for (int i = 0; i < kWaitPolls; ++i)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}

// ----------------------------------------------------------- conversions
template <class R>
__device__ __forceinline__ R to_r(double v) { return static_cast<R>(v); }

__device__ __forceinline__ float bf2f(bf16 v) { return __bfloat162float(v); }

// Load VL consecutive complex numbers (re, im interleaved) starting at p.
template <class S, int VL, class R>
__device__ __forceinline__ void load_lanes(const S* __restrict__ p, R* re, R* im) {
    if constexpr (std::is_same<S, double>::value) {
#pragma unroll
        for (int v = 0; v < VL; ++v) {
            double2 t = reinterpret_cast<const double2*>(p)[v];
            re[v] = (R)t.x;
            im[v] = (R)t.y;
        }
    } else if constexpr (std::is_same<S, float>::value) {
        if constexpr (VL % 2 == 0) {
#pragma unroll
            for (int v = 0; v < VL; v += 2) {
                float4 t = reinterpret_cast<const float4*>(p)[v / 2];
                re[v] = (R)t.x; im[v] = (R)t.y; re[v + 1] = (R)t.z; im[v + 1] = (R)t.w;
            }
        } else {
#pragma unroll
            for (int v = 0; v < VL; ++v) {
                float2 t = reinterpret_cast<const float2*>(p)[v];
                re[v] = (R)t.x; im[v] = (R)t.y;
            }
        }
    } else {  // bf16
        if constexpr (VL % 4 == 0) {
#pragma unroll
            for (int v = 0; v < VL; v += 4) {
                uint4 t = reinterpret_cast<const uint4*>(p)[v / 4];
                const __nv_bfloat162* q = reinterpret_cast<const __nv_bfloat162*>(&t);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float2 f = __bfloat1622float2(q[j]);
                    re[v + j] = (R)f.x; im[v + j] = (R)f.y;
                }
            }
        } else if constexpr (VL % 2 == 0) {
#pragma unroll
            for (int v = 0; v < VL; v += 2) {
                uint2 t = reinterpret_cast<const uint2*>(p)[v / 2];
                const __nv_bfloat162* q = reinterpret_cast<const __nv_bfloat162*>(&t);
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    float2 f = __bfloat1622float2(q[j]);
                    re[v + j] = (R)f.x; im[v + j] = (R)f.y;
                }
            }
        } else {
#pragma unroll
            for (int v = 0; v < VL; ++v) {
                __nv_bfloat162 q = reinterpret_cast<const __nv_bfloat162*>(p)[v];
                float2 f = __bfloat1622float2(q);
                re[v] = (R)f.x; im[v] = (R)f.y;
            }
        }
    }
}

// Store VL consecutive complex numbers; CS = true uses the cache-streaming
// hint (data written once and not re-read by this kernel: keep it from
// evicting re-used lines in L2).
template <class S, int VL, class R, bool CS = false>
__device__ __forceinline__ void store_lanes(S* __restrict__ p, const R* re, const R* im) {
    if constexpr (std::is_same<S, double>::value) {
#pragma unroll
        for (int v = 0; v < VL; ++v) {
            const double2 t = make_double2((double)re[v], (double)im[v]);
            if (CS) __stcs(reinterpret_cast<double2*>(p) + v, t);
            else reinterpret_cast<double2*>(p)[v] = t;
        }
    } else if constexpr (std::is_same<S, float>::value) {
        if constexpr (VL % 2 == 0) {
#pragma unroll
            for (int v = 0; v < VL; v += 2) {
                const float4 t = make_float4((float)re[v], (float)im[v], (float)re[v + 1], (float)im[v + 1]);
                if (CS) __stcs(reinterpret_cast<float4*>(p) + v / 2, t);
                else reinterpret_cast<float4*>(p)[v / 2] = t;
            }
        } else {
#pragma unroll
            for (int v = 0; v < VL; ++v) {
                const float2 t = make_float2((float)re[v], (float)im[v]);
                if (CS) __stcs(reinterpret_cast<float2*>(p) + v, t);
                else reinterpret_cast<float2*>(p)[v] = t;
            }
        }
    } else {
        if constexpr (VL % 4 == 0) {
#pragma unroll
            for (int v = 0; v < VL; v += 4) {
                uint4 t;
                __nv_bfloat162* q = reinterpret_cast<__nv_bfloat162*>(&t);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    q[j] = __floats2bfloat162_rn((float)re[v + j], (float)im[v + j]);
                if (CS) __stcs(reinterpret_cast<uint4*>(p) + v / 4, t);
                else reinterpret_cast<uint4*>(p)[v / 4] = t;
            }
        } else if constexpr (VL % 2 == 0) {
#pragma unroll
            for (int v = 0; v < VL; v += 2) {
                uint2 t;
                __nv_bfloat162* q = reinterpret_cast<__nv_bfloat162*>(&t);
#pragma unroll
                for (int j = 0; j < 2; ++j)
                    q[j] = __floats2bfloat162_rn((float)re[v + j], (float)im[v + j]);
                if (CS) __stcs(reinterpret_cast<uint2*>(p) + v / 2, t);
                else reinterpret_cast<uint2*>(p)[v / 2] = t;
            }
        } else {
#pragma unroll
            for (int v = 0; v < VL; ++v)
                reinterpret_cast<__nv_bfloat162*>(p)[v] =
                    __floats2bfloat162_rn((float)re[v], (float)im[v]);
        }
    }
}

// One complex number.
template <class S, class R>
__device__ __forceinline__ void load_c1(const S* p, R& re, R& im) {
    R a[1], b[1];
    load_lanes<S, 1, R>(p, a, b);
    re = a[0];
    im = b[0];
}

// Link element (re, im) of precision SL as R.
template <class SL, class R>
__device__ __forceinline__ void link_c(const SL* w, int idx, R& re, R& im) {
    if constexpr (std::is_same<SL, bf16>::value) {
        float2 f = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(w)[idx]);
        re = (R)f.x;
        im = (R)f.y;
    } else {
        re = (R)w[2 * idx];
        im = (R)w[2 * idx + 1];
    }
}

// Deterministic block reduction of one double per thread into per-rhs sums.
// vals: shared scratch of blockDim.x doubles; rhs_of(t) gives the rhs of
// thread t (or -1).  Result written by warp w for rhs r = w, w + nwarps, ...
template <class RhsOf>
__device__ __forceinline__ void block_rhs_reduce(double v, double* vals, int nrhs, RhsOf rhs_of,
                                                 double* out /* [nrhs] */) {
    vals[threadIdx.x] = v;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    for (int r = warp; r < nrhs; r += nwarps) {
        double s = 0.0;
        for (int t = lane; t < (int)blockDim.x; t += 32)
            if (rhs_of(t) == r) s += vals[t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) out[r] = s;
    }
    __syncthreads();
}

}  // namespace dwf
