// The energy-weighted DOA error of Section 4 (Eq. 16-20) on the device:
//   RMSE_alpha = || sum_l f_alpha(s_qbar_l) Y_l / sum_l Y_l - f_alpha(s_0) ||_2
// over the frames l of one configuration, s_qbar_l the chosen direction (unit vector of grid
// point idx[l]), Y_l its energy (Algorithm 1's online step 4 score).  f_1 maps a direction to
// the arc [cos g, 0, sin g], g = atan2(s_z, sqrt(s_x^2 + s_y^2)) (Eq. 16, 17); f_2 to the upper
// hemisphere [s_x, s_y, |s_z|] (Eq. 18); f_3 is the identity (Eq. 19).  One CTA sums in FP64 in
// a fixed order (thread-strided partial sums, then a tree), so the result is reproducible.
// Frames with idx < 0 or a non-finite Y are left out.
#include <cuda_runtime.h>
#include <math.h>

#include <cmath>

#include "common.h"

namespace sp {
namespace {

constexpr int kRmseThreads = 256;

__device__ __forceinline__ void doa_map(int alpha, double x, double y, double z, double *f) {
    if (alpha == 1) {
        const double g = atan2(z, sqrt(x * x + y * y));
        f[0] = cos(g);
        f[1] = 0.0;
        f[2] = sin(g);
    } else if (alpha == 2) {
        f[0] = x;
        f[1] = y;
        f[2] = fabs(z);
    } else {
        f[0] = x;
        f[1] = y;
        f[2] = z;
    }
}

__global__ void __launch_bounds__(kRmseThreads)
    weighted_doa_kernel(const double *__restrict__ dirs, const int32_t *__restrict__ idx, const float *__restrict__ Y,
                        int T, int alpha, double *__restrict__ out4) {
    __shared__ double red[4][kRmseThreads];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};   // sum f Y (3), sum Y
    for (int l = threadIdx.x; l < T; l += blockDim.x) {
        const int q = idx[l];
        const float y = Y[l];
        if (q < 0 || !isfinite(y)) continue;
        double f[3];
        doa_map(alpha, dirs[3 * q], dirs[3 * q + 1], dirs[3 * q + 2], f);
        acc[0] += f[0] * (double)y;
        acc[1] += f[1] * (double)y;
        acc[2] += f[2] * (double)y;
        acc[3] += (double)y;
    }
    for (int c = 0; c < 4; ++c) red[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int h = kRmseThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 4) out4[threadIdx.x] = red[threadIdx.x][0];
}

}  // namespace
}  // namespace sp

using namespace sp;

extern "C" int sp_weighted_doa_error(const sp_steering *st, const int32_t *idx_dev, const float *score_dev, int T,
                                     const double *s0, int alpha, double *rmse_out, void *stream) {
    SP_CHECK(st && s0 && rmse_out, SP_EINVAL, "sp_weighted_doa_error: null pointer");
    SP_CHECK(alpha >= 1 && alpha <= 3, SP_EINVAL, "sp_weighted_doa_error: alpha must be 1, 2 or 3");
    SP_CHECK(T >= 1 && T <= (1 << 28), SP_EINVAL, "sp_weighted_doa_error: T out of range");
    SP_CHECK(idx_dev && score_dev && (reinterpret_cast<uintptr_t>(idx_dev) & 3) == 0 &&
                 (reinterpret_cast<uintptr_t>(score_dev) & 3) == 0,
             SP_EINVAL, "sp_weighted_doa_error: idx_dev / score_dev NULL or misaligned");
    const double n0 = std::sqrt(s0[0] * s0[0] + s0[1] * s0[1] + s0[2] * s0[2]);
    SP_CHECK(std::isfinite(n0) && n0 > 0, SP_EINVAL, "sp_weighted_doa_error: s0 must be a nonzero direction");
    double *d_out = nullptr;
    SP_CUDA(cudaMalloc(&d_out, 4 * sizeof(double)));
    cudaStream_t s = (cudaStream_t)stream;
    weighted_doa_kernel<<<1, kRmseThreads, 0, s>>>(st->d_dirs.as<double>(), idx_dev, score_dev, T, alpha, d_out);
    double h[4] = {0, 0, 0, 0};
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d_out, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_out);
    SP_CHECK(e == cudaSuccess, SP_ECUDA, std::string("sp_weighted_doa_error: ") + cudaGetErrorString(e));
    SP_CHECK(h[3] != 0.0, SP_EINVAL, "sp_weighted_doa_error: the energies sum to zero");
    // f_alpha(s0) of the unit direction, on the host with the same formulas
    const double u[3] = {s0[0] / n0, s0[1] / n0, s0[2] / n0};
    double f0[3];
    if (alpha == 1) {
        const double g = std::atan2(u[2], std::sqrt(u[0] * u[0] + u[1] * u[1]));
        f0[0] = std::cos(g);
        f0[1] = 0.0;
        f0[2] = std::sin(g);
    } else if (alpha == 2) {
        f0[0] = u[0];
        f0[1] = u[1];
        f0[2] = std::fabs(u[2]);
    } else {
        f0[0] = u[0];
        f0[1] = u[1];
        f0[2] = u[2];
    }
    double r2 = 0.0;
    for (int c = 0; c < 3; ++c) {
        const double d = h[c] / h[3] - f0[c];
        r2 += d * d;
    }
    *rmse_out = std::sqrt(r2);
    return SP_OK;
}
