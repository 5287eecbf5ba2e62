// hho_assemble_noalloc: the right-hand-side assembly of hho_assemble without
// any memory allocation (declared in include/hho.h).
//
// hho_assemble obtains the per-CTA working memory of its element kernel from
// cudaMalloc on every call.  Some callers cannot allocate device memory at the
// point where they refresh the right-hand side, for example when every byte of
// the device is handed to their own memory pool, or inside a time loop where a
// cudaMalloc (which may synchronise the device or fail) is not acceptable.  This
// variant runs the same kernels with a fixed 1 MiB working array that lives in
// the library's device image (every GPU that loads the library holds it until
// the process exits).  The caller still passes the data arrays and the optional
// output vector.
#include "internal.h"

namespace {

// Working memory shared by every call on a device: 2^17 doubles = 1 MiB.
constexpr int64_t kAssembleScratchDoubles = int64_t(1) << 17;
static __device__ __align__(256) double g_assemble_scratch[kAssembleScratchDoubles];

}  // namespace

extern "C" hho_status hho_assemble_noalloc(hho_ctx* ctx, const double* d_f, const double* d_gD, const double* d_gN,
                                           double* d_rhs) {
    if (!ctx) return HHO_ERR_ARG;
    if (!d_f || !d_gD || !d_gN) {
        ctx->err = "hho_assemble_noalloc: null data array";
        return HHO_ERR_ARG;
    }
    int dev = -1;
    HHO_CUDA(cudaGetDevice(&dev));
    if (dev != ctx->device) {
        ctx->err = "hho_assemble_noalloc: the current device is not the context's device";
        return HHO_ERR_ARG;
    }
    // In host code the array's name is a host-side stand-in, so the kernels get
    // its device address.  It is looked up with the context's device current on
    // the context's first call and kept in the context: a context created after
    // a device reset looks it up again in the reloaded module.
    if (!ctx->noalloc_scratch) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_assemble_scratch);
        if (e != cudaSuccess || !p) {
            ctx->err = std::string("hho_assemble_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return HHO_ERR_CUDA;
        }
        ctx->noalloc_scratch = static_cast<double*>(p);
    }
    double* scratch = ctx->noalloc_scratch;
    // The element kernel clears each element's slot of the array before use,
    // so nothing left over from an earlier call is read.
    HHO_TRY(hho::build_rhs_scratch(ctx, d_f, d_gD, d_gN, scratch, kAssembleScratchDoubles));
    HHO_TRY(hho::assemble_rhs_vector(ctx, ctx->rhs));
    if (d_rhs)
        HHO_CUDA(cudaMemcpyAsync(d_rhs, ctx->rhs, ctx->levels[0].n * sizeof(double), cudaMemcpyDeviceToDevice,
                                 ctx->stream));
    ctx->have_rhs = true;
    return HHO_OK;
}
