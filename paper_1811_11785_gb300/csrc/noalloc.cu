// sp_localize_noalloc: the FP16/BF16 exhaustive localisation (the same kernels as
// sp_localize with SP_MODE_SVD_EXHAUSTIVE) with its scratch memory -- the per-frame Z
// vectors and their squared norms -- in a fixed array compiled into this library, so that
// the call itself allocates nothing.  It exists for callers that must not enter the CUDA
// allocator on their processing path: real-time audio callbacks and plugin hosts, where
// cudaMalloc can block on driver locks and stall the audio deadline, and deployments whose
// device memory budget is fixed when the process starts.
#include <cuda_runtime.h>

#include <mutex>

#include "common.h"

namespace sp {

// 8 MiB, 256-byte aligned; every GPU that loads this library holds it until exit.
constexpr size_t kNoAllocBytes = size_t(8) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The name of a __device__
// array is only a host-side stand-in, so the address is looked up once per device (with
// that device current) and cached.
static int noalloc_scratch(void **out) {
    int dev = 0;
    SP_CUDA(cudaGetDevice(&dev));
    SP_CHECK(dev >= 0 && dev < kMaxDevices, SP_ENOTIMPL, "sp_localize_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            return fail(SP_ECUDA, std::string("sp_localize_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return SP_OK;
}

}  // namespace sp

using namespace sp;

extern "C" int sp_localize_noalloc(const sp_basis *b, const void *frames_dev, int T, sp_prec prec,
                                   int32_t *idx_dev, float *score_dev, float *proj_score_dev, void *stream) {
    // the same argument checks as sp_localize (frames, T range, output pointers and alignment)
    SP_TRY(check_localize_args(b, frames_dev, T, idx_dev, score_dev, proj_score_dev));
    SP_CHECK(prec == SP_PREC_FP16 || prec == SP_PREC_BF16, SP_ENOTIMPL,
             "sp_localize_noalloc: only SP_PREC_FP16 and SP_PREC_BF16");
    SP_CHECK(b->tc.n1 > 0 && b->tc_maps, SP_ENOTIMPL,
             "sp_localize_noalloc: the tensor-core path supports 2K <= 288 and M <= 16");
    const size_t zbytes = ((size_t)T * b->K * 8 + 255) / 256 * 256;
    const size_t nbytes = ((size_t)T * 4 + 255) / 256 * 256;
    const size_t need = zbytes + nbytes + scan_workspace_bytes(T);
    SP_CHECK(need <= kNoAllocBytes, SP_EINVAL,
             "sp_localize_noalloc: about T * (8 K + 16) bytes of scratch exceeds the built-in 8 MiB (" +
                 std::to_string(need) + " bytes requested)");
    void *scratch = nullptr;
    SP_TRY(noalloc_scratch(&scratch));
    if (T == 0) {
        // the warm-up call: with the scratch address cached above, load every kernel a call on
        // this basis can launch and set their shared-memory limits, so that later calls do
        // neither on the caller's processing path
        SP_TRY(prepare_tc(b, (int)prec));
        SP_TRY(prepare_simt(b->st));
        return prepare_step4(b->st);
    }
    char *z = static_cast<char *>(scratch);
    float *zn2 = reinterpret_cast<float *>(z + zbytes);
    cudaStream_t s = (cudaStream_t)stream;
    SP_TRY(launch_svd_proj(b, frames_dev, T, (int)prec, z, zn2, s));
    SP_TRY(launch_svd_scan(b, z, zn2, T, (int)prec, idx_dev, proj_score_dev, s, z + zbytes + nbytes));
    if (score_dev) SP_TRY(launch_score_row(b->st, frames_dev, T, idx_dev, score_dev, s));
    return SP_OK;
}
