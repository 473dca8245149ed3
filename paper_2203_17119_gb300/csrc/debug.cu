// The debug build (-DDWF_DEBUG, libdwf_debug.so): host-side bounds checks in
// the entry points.  Every caller buffer an entry point reads or writes is
// checked, before anything is launched, to lie inside one device allocation
// of the current context ([p, p + bytes) within the range the CUDA driver reports
// for p); the handle's neighbour and link tables are checked when they are
// built.  Failures return DWF_ERR_ARG with the buffer's name.  With a caching
// allocator (PyTorch's) the allocation is the allocator's segment, so only
// overruns past the segment are caught; PYTORCH_NO_CUDA_MEMORY_CACHING=1 makes
// every tensor its own allocation.  In the release build the checks compile
// to nothing and dwf_check_range reports DWF_ERR_UNSUPPORTED.
#include <cstdint>
#include <initializer_list>
#include <mutex>

#include "dwf_internal.cuh"

namespace dwf {

size_t field_bytes(const dwf_handle* h, int kind, dwf_prec prec, int nrhs) {
    if (h == nullptr || nrhs < 1 || nrhs > h->nrhs_max || (prec != DWF_FP64 && prec != DWF_FP32 && prec != DWF_BF16))
        return 0;
    const int64_t sites = kind == 2 ? h->nsite[0] + h->nsite[1] : h->nsite[kind & 1];
    const size_t complex_bytes = prec == DWF_FP64 ? 16 : prec == DWF_FP32 ? 8 : 4;
    return (size_t)sites * 12 * h->p.Ls * nrhs * complex_bytes;
}

size_t link_field_bytes(const dwf_handle* h) {
    return (size_t)h->p.dims[0] * h->p.dims[1] * h->p.dims[2] * h->p.dims[3] * 4 * 9 * 16;
}

#ifdef DWF_DEBUG
namespace {
typedef int (*AddressRangeFn)(unsigned long long*, size_t*, unsigned long long);
AddressRangeFn address_range() {
    static AddressRangeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<AddressRangeFn>(f);
    });
    return fn;
}
}  // namespace

dwf_status debug_range(const void* p, size_t bytes, const char* who, const char* what) {
    if (p == nullptr || bytes == 0) return DWF_OK;   // the entry point's own checks report these
    AddressRangeFn fn = address_range();
    if (fn == nullptr) {
        set_error("%s: the debug build cannot query device allocation ranges", who);
        return DWF_ERR_CUDA;
    }
    unsigned long long base = 0;
    size_t size = 0;
    const unsigned long long a = (unsigned long long)(uintptr_t)p;
    if (fn(&base, &size, a) != 0) {
        set_error("%s: %s (%p) is not device memory of the current context", who, what, p);
        return DWF_ERR_ARG;
    }
    if (a + bytes > base + size) {
        set_error("%s: %s needs %zu bytes but its allocation ends %llu bytes after it", who, what, bytes,
                  (unsigned long long)(base + size - a));
        return DWF_ERR_ARG;
    }
    return DWF_OK;
}

dwf_status debug_ranges(const char* who, std::initializer_list<FieldRange> r) {
    for (const FieldRange& f : r) DWF_TRY(debug_range(f.p, f.bytes, who, f.what));
    return DWF_OK;
}
#endif

}  // namespace dwf

extern "C" {

dwf_status dwf_debug_build(int* on) {
    if (on == nullptr) {
        dwf::set_error("dwf_debug_build: null output");
        return DWF_ERR_ARG;
    }
#ifdef DWF_DEBUG
    *on = 1;
#else
    *on = 0;
#endif
    return DWF_OK;
}

dwf_status dwf_check_range(const void* p, size_t bytes) {
#ifdef DWF_DEBUG
    if (p == nullptr || bytes == 0) {
        dwf::set_error("dwf_check_range: null pointer or zero size");
        return DWF_ERR_ARG;
    }
    return dwf::debug_range(p, bytes, "dwf_check_range", "the buffer");
#else
    (void)p;
    (void)bytes;
    dwf::set_error("dwf_check_range: the library was built without DWF_DEBUG");
    return DWF_ERR_UNSUPPORTED;
#endif
}

}  // extern "C"
