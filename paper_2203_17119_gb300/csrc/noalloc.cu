// dwf_mpc_noalloc: the Schur operator M_pc with its two checkerboard
// temporaries taken from a file-scope static device array instead of the
// handle's scratch buffers.
//
// Who needs it: code that may not call cudaMalloc on the path where it
// applies the operator -- a host framework that owns all device memory
// through its own pool and forbids raw allocations, or an embedding that
// must keep the footprint of its calls fixed and known at load time.
// The array below is reserved when the module loads, on every GPU that loads
// the library, and is held until the process exits.
//
// Limits and sharing: each of the two temporaries holds at most
// kNoAllocTempBytes (32 MiB), i.e. max(n_even, n_odd) * 12 * Ls * nrhs
// complex numbers of the chosen precision; larger requests fail with
// DWF_ERR_ARG.  Every call on a device shares the same array and it keeps the
// last call's contents; both temporaries are fully written before they are
// read, so nothing has to start at zero.  Calls whose kernels overlap on the
// GPU (different streams, or different handles on concurrent streams) race
// on the array: serialise them.
//
// Set-up: the first call on a device, with that device current, looks up the
// array's device address with cudaGetSymbolAddress and caches it; make that
// first call before any stream capture.
#include <mutex>

#include "dev_common.cuh"
#include "dwf_internal.cuh"

namespace dwf {

constexpr size_t kNoAllocTempBytes = (size_t)32 << 20;
constexpr int kNoAllocMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[2 * kNoAllocTempBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[kNoAllocMaxDevices] = {};

static dwf_status noalloc_scratch(void** out) {
    int dev = 0;
    DWF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("dwf_mpc_noalloc: device ordinal %d out of range", dev);
        return DWF_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_addr[dev] == nullptr) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_error("dwf_mpc_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return DWF_ERR_CUDA;
        }
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return DWF_OK;
}

}  // namespace dwf

using namespace dwf;

extern "C" dwf_status dwf_mpc_noalloc(dwf_handle* h, void* out, const void* in, int dagger,
                                      dwf_prec prec, int nrhs, void* stream) {
    DWF_RANGE("dwf_mpc_noalloc");
    DWF_TRY(check_handle(h));
    if (out == nullptr || in == nullptr || out == in) {
        set_error("dwf_mpc_noalloc: null or aliasing field pointers");
        return DWF_ERR_ARG;
    }
    if (prec != DWF_FP64 && prec != DWF_FP32 && prec != DWF_BF16) {
        set_error("dwf_mpc_noalloc: bad precision %d", (int)prec);
        return DWF_ERR_ARG;
    }
    if (nrhs < 1 || nrhs > h->nrhs_max) {
        set_error("dwf_mpc_noalloc: nrhs = %d outside [1, %d]", nrhs, h->nrhs_max);
        return DWF_ERR_ARG;
    }
    if (!h->have_gauge) {
        set_error("dwf_mpc_noalloc: no gauge field loaded (dwf_set_gauge)");
        return DWF_ERR_ARG;
    }
    const size_t nmax = cb_elems(h, 0, nrhs) > cb_elems(h, 1, nrhs) ? cb_elems(h, 0, nrhs)
                                                                    : cb_elems(h, 1, nrhs);
    const size_t need = nmax * 2 * prec_size(prec);
    if (need > kNoAllocTempBytes) {
        set_error("dwf_mpc_noalloc: needs %zu bytes per temporary; the static scratch holds %zu",
                  need, kNoAllocTempBytes);
        return DWF_ERR_ARG;
    }
    // the tile table must already exist: building one would allocate (the
    // same tile size the launches below look up)
    if (find_tiles(h, tile_or_default(tile_for(h, nrhs))) == nullptr) {
        set_error("dwf_mpc_noalloc: no tile table for nrhs = %d yet (call dwf_mpc or dwf_autotune "
                  "once first)", nrhs);
        return DWF_ERR_ARG;
    }
    void* base = nullptr;
    DWF_TRY(noalloc_scratch(&base));
    unsigned char* tA = static_cast<unsigned char*>(base);
    unsigned char* tB = tA + kNoAllocTempBytes;
    return op_mpc(h, out, in, dagger ? 1 : 0, prec, prec, nrhs, tA, tB, nullptr, nullptr,
                  (cudaStream_t)stream);
}
