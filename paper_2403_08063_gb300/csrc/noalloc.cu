// mg_exchange_level_noalloc: the one-level ghost exchange of mg_exchange_level without any device allocation.
//
// mg_exchange_level allocates (cudaMalloc) a padded scratch pool for the level on every call and frees it
// afterwards.  Some callers cannot let a library allocate device memory at that point: applications whose device
// memory is entirely handed to a caching allocator or reserved at start-up (a cudaMalloc then fails or steals
// from the pool), and loops with a latency budget that must not enter CUDA's device allocator (cudaMalloc and
// cudaFree can synchronise the device and take unbounded time).  They use this variant.  Its scratch pool is the
// file-scope device array below, of a fixed size; every GPU that loads the library holds that array until the
// process exits.  The call allocates nothing else either: on a forest whose FP64 face coefficients do not exist
// yet (variable k with FP32 cycles creates them on first use) it returns MG_ERR_STATE instead of creating them.
#include <mutex>

#include "forest_state.h"

// 4 MiB of FP64 scratch: enough for levels with nb * (n+2)^3 (rounded to 32 elements per block) <= 524,288,
// e.g. 8 blocks of 64^3 or 120 blocks of 16^3 (the refined 56 + 64 block forest at 16^3 cells).
constexpr int64_t kScratchElems = 524288;
static __device__ __align__(256) double g_exchange_scratch[kScratchElems];

namespace octmg {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
double *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code the array's name is only a host-side
// stand-in, so the address is looked up once per device (with that device current) and cached.
mg_status scratch_address(double **out) {
    int dev = 0;
    MG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("mg_exchange_level_noalloc: device index out of range");
        return MG_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        MG_CUDA(cudaGetSymbolAddress(&p, g_exchange_scratch));
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return MG_OK;
}

}  // namespace
}  // namespace octmg

using namespace octmg;

extern "C" mg_status mg_exchange_level_noalloc(mg_forest *F, int32_t level, const double *u_dev, double *padded_dev) {
    if (!F || !u_dev || !padded_dev || level < 0 || level >= static_cast<int32_t>(F->L.size())) {
        set_error("bad argument");
        return MG_ERR_INVALID_ARG;
    }
    if (F->cfg.coeff && !F->rhs_set) {
        set_error("mg_set_rhs (k) has not been called");
        return MG_ERR_STATE;
    }
    DevLevel &d = F->L[level];
    // The conservative fine-to-coarse ghosts of a variable-k forest read the level's FP64 face coefficients.  A
    // forest with FP32 cycles creates those arrays lazily (cudaMalloc), which this entry point must not do.
    if (F->cfg.coeff && F->cfg.interface_flux && d.nsegs && (!d.tx || !d.ty || !d.tz)) {
        set_error("mg_exchange_level_noalloc: the FP64 face coefficients of level " + std::to_string(level) +
                  " do not exist yet (a variable-k forest with FP32 cycles creates them on first use, which "
                  "allocates); call mg_exchange_level, mg_apply or mg_adjoint_solve once first");
        return MG_ERR_STATE;
    }
    const int64_t need = d.pool_elems();
    if (need > kScratchElems) {
        set_error("mg_exchange_level_noalloc: level " + std::to_string(level) + " needs " + std::to_string(need) +
                  " doubles of scratch, more than the " + std::to_string(kScratchElems) +
                  " of the static scratch array; use mg_exchange_level");
        return MG_ERR_INVALID_ARG;
    }
    double *pool = nullptr;
    MG_TRY(scratch_address(&pool));
    // The array keeps the previous call's contents: clear the part this level uses, so the edge and corner ghosts
    // (which no exchange writes) read 0 as in mg_exchange_level.
    MG_CUDA(cudaMemsetAsync(pool, 0, need * sizeof(double), F->st));
    k_pack<double><<<grid_for(d.cells()), kThreads, 0, F->st>>>(pool, u_dev, d.g);
    exchange_any64(F, d, pool);
    const size_t per = static_cast<size_t>(d.g.P) * d.g.P * d.g.P;
    MG_CUDA(cudaMemcpy2DAsync(padded_dev, per * sizeof(double), pool, d.g.bs * sizeof(double), per * sizeof(double),
                              d.g.nb, cudaMemcpyDeviceToDevice, F->st));
    MG_CUDA(cudaStreamSynchronize(F->st));
    return MG_OK;
}
