// Chebyshev filter of the normal Schur operator, the recursively built filter
// functions proposed in Sec. 4 for a fast multigrid set-up of the local
// (D_Omega) solves:
//
//   out = T_n(z(A)) in,   A = M_pc^+ M_pc,   z(lam) = (hi + lo - 2 lam) / (hi - lo),
//
// by the three-term recurrence w_{k+1} = 2 z(A) w_k - w_{k-1} (w_0 = in,
// w_1 = z(A) in).  Each step is M_pc, M_pc^+ (the operator kernels, FP64 or
// FP32) and two axpby passes; on a box handle every box is filtered with its
// own Dirichlet operator at once.
#include "dwf_internal.cuh"

namespace dwf {

dwf_status chebyshev_filter(dwf_handle* h, void* out, const void* in, int order, double lo, double hi,
                            dwf_prec prec, int nrhs, cudaStream_t s) {
    if (!h->have_gauge) {
        set_error("chebyshev: no gauge field loaded");
        return DWF_ERR_ARG;
    }
    if (out == nullptr || in == nullptr || out == in || nrhs < 1 || nrhs > h->nrhs_max || order < 0 ||
        !(hi > lo) || (prec != DWF_FP64 && prec != DWF_FP32)) {
        set_error("chebyshev: bad arguments (distinct odd cb fields, 1 <= nrhs <= nrhs_max, order >= 0, "
                  "hi > lo, FP64 or FP32)");
        return DWF_ERR_ARG;
    }
    const size_t bytes = cb_elems(h, 1, nrhs) * prec_size(prec) * 2;
    DWF_CUDA(cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, s));
    if (order == 0) return DWF_OK;
    const double c0 = (hi + lo) / (hi - lo), c1 = -2.0 / (hi - lo);
    const int T = tile_for(h, nrhs);
    char* scratch = nullptr;   // three fields: w_{k-1}, M_pc w_k, A w_k
    DWF_CUDA(dev_malloc(&scratch, 3 * bytes));
    void* a = scratch;
    void* u = scratch + bytes;
    void* t = scratch + 2 * bytes;
    auto A = [&](void* dst, const void* src) -> dwf_status {
        DWF_TRY(op_mpc(h, u, src, 0, prec, prec, nrhs, h->d_tmp, h->d_tmp2, nullptr, nullptr, s));
        return op_mpc(h, dst, u, 1, prec, prec, nrhs, h->d_tmp, h->d_tmp2, nullptr, nullptr, s);
    };
    auto run = [&]() -> dwf_status {
        // a = w_0 = in, b = w_1 = c0 in + c1 A in (b lives in out)
        DWF_CUDA(cudaMemcpyAsync(a, in, bytes, cudaMemcpyDeviceToDevice, s));
        DWF_TRY(A(t, in));
        DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, c1, t, prec, nullptr, c0, out, prec, nullptr, T, s));
        void* b = out;
        for (int k = 1; k < order; ++k) {
            // a <- 2 c0 b + 2 c1 A b - a = w_{k+1}; then swap the roles of a and b
            DWF_TRY(A(t, b));
            DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, 2.0 * c0, b, prec, nullptr, -1.0, a, prec, nullptr, T, s));
            DWF_TRY(launch_axpby(h, 1, nrhs, nullptr, 2.0 * c1, t, prec, nullptr, 1.0, a, prec, nullptr, T, s));
            void* tmp = a;
            a = b;
            b = tmp;
        }
        if (b != out) DWF_CUDA(cudaMemcpyAsync(out, b, bytes, cudaMemcpyDeviceToDevice, s));
        return DWF_OK;
    };
    const dwf_status st = run();
    cudaStreamSynchronize(s);
    cudaFree(scratch);
    return st;
}

}  // namespace dwf
