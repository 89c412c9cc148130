// The STFT front end of Section 2 and the binary time-frequency mask of the paper's conclusion.
//
// X_m^l[k] = sum_{n<N} w[n] x_m[l dN + n] exp(-2 pi i k n / N), k = 0 .. N/2, with the sine
// window w[n] = sin(pi (n + 1/2) / N).  Each transform is a real N-point DFT computed as an
// N/2-point complex FFT of z[j] = (w x)[2j] + i (w x)[2j + 1] (radix-2 Stockham in shared
// memory, natural order out), followed by X[k] = E[k] + exp(-2 pi i k / N) O[k] with
// E[k] = (Z[k] + conj(Z[N/2 - k])) / 2 and O[k] = (Z[k] - conj(Z[N/2 - k])) / (2i), the DFTs of
// the even and odd samples.  A CTA takes `fpc` frames x M channels at a time (persistent grid);
// the samples of a frame are read coalesced from the channel rows, the bins written coalesced
// in the [T][M][B] layout the localisation calls take; window and twiddles come from tables
// the CTA computes once in shared memory.
//
// Mask: where mask[l][k] is 0 the bin of every channel is written as 0.  A zero spectrum entry
// is a zero cross spectrum under Eq. 3's |X|^2 < 1e-30 rule, so a masked bin drops out of every
// SRP-PHAT and SVD-PHAT score (Eq. 5, 9, 12, 14) and of online step 4.
#include <cuda_runtime.h>
#include <math.h>

#include "common.h"
#include "debug.cuh"

namespace sp {
namespace {

constexpr int kStftThreads = 256;
constexpr int kStftPoints = 2048;   // complex points per CTA (all its transforms), per buffer

// Persistent: a CTA takes groups of `fpc` frames x M channels in turn.  Shared memory: two
// buffers of fpc M n complex points, then the tables the CTA computes once: the window w[N],
// the stage twiddles exp(-2 pi i j / n) for j < n/2, and the post-processing twiddles
// exp(-2 pi i k / N) for k <= n.
__global__ void __launch_bounds__(kStftThreads)
    stft_kernel(const float *__restrict__ x, long long ld, int M, int N, int lg_n, int hop, int T, int fpc,
                const uint8_t *__restrict__ mask, float2 *__restrict__ out, int *status) {
    extern __shared__ float2 sbuf[];
    const int n = N / 2, B = n + 1, hn = n / 2;
    const int G = fpc * M;                       // transforms per group
    float2 *buf0 = sbuf, *buf1 = sbuf + G * n;
    float2 *tw = buf1 + G * n;                   // [n/2]
    float2 *pt = tw + (hn > 0 ? hn : 1);         // [n + 1]
    float *win = reinterpret_cast<float *>(pt + B);   // [N]
    for (int j = threadIdx.x; j < hn; j += blockDim.x) {
        float s, c;
        sincospif(-2.f * (float)j / (float)n, &s, &c);
        tw[j] = make_float2(c, s);
    }
    for (int k = threadIdx.x; k < B; k += blockDim.x) {
        float s, c;
        sincospif(-2.f * (float)k / (float)N, &s, &c);
        pt[k] = make_float2(c, s);
    }
    for (int t = threadIdx.x; t < N; t += blockDim.x) win[t] = sinpif(((float)t + 0.5f) / (float)N);
    __syncthreads();
    const int n_groups = (int)(((long long)T + fpc - 1) / fpc);
    for (int grp = blockIdx.x; grp < n_groups; grp += gridDim.x) {
        const long long l0 = (long long)grp * fpc;
        float2 *src = buf0, *dst = buf1;
        // load: z[g][j] = (w x)[2j] + i (w x)[2j + 1], transform g = (frame l0 + g / M, channel g % M)
        for (int g = 0; g < G; ++g) {
            const long long l = l0 + g / M;
            const int m = g % M;
            const float *row = x + (size_t)m * ld + (size_t)l * hop;
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                float2 v = make_float2(0.f, 0.f);
                if (l < T && dcheck((long long)l * hop + 2 * j + 1 < ld, status))
                    v = make_float2(win[2 * j] * row[2 * j], win[2 * j + 1] * row[2 * j + 1]);
                src[g * n + j] = v;
            }
        }
        __syncthreads();
        // radix-2 Stockham: stage of half-length L maps a, b = src[i], src[i + n/2] to
        // dst[2j + k] = a + w b, dst[2j + k + L] = a - w b with k = i mod L, j = i - k,
        // w = exp(-i pi k / L) = tw[k n / (2L)]
        for (int L = 1, lg = 0; L < n; L <<= 1, ++lg) {
            const int shift = lg_n - 1 - lg;         // k n / (2L) = k << shift
            for (int e = threadIdx.x; e < G * hn; e += blockDim.x) {
                const int g = e >> (lg_n - 1), i = e & (hn - 1);
                const int k = i & (L - 1), j = i - k;
                const float2 a = src[g * n + i], b = src[g * n + i + hn];
                const float2 w = tw[k << shift];
                const float2 wb = make_float2(w.x * b.x - w.y * b.y, w.x * b.y + w.y * b.x);
                dst[g * n + 2 * j + k] = make_float2(a.x + wb.x, a.y + wb.y);
                dst[g * n + 2 * j + k + L] = make_float2(a.x - wb.x, a.y - wb.y);
            }
            __syncthreads();
            float2 *t = src;
            src = dst;
            dst = t;
        }
        // real-input post-processing and the store (with the mask)
        for (int g = 0; g < G; ++g) {
            const long long l = l0 + g / M;
            if (l >= T) break;
            const int m = g % M;
            const uint8_t *mrow = mask ? mask + (size_t)l * B : nullptr;
            float2 *orow = out + ((size_t)l * M + m) * B;
            for (int k = threadIdx.x; k < B; k += blockDim.x) {
                const float2 zk = src[g * n + (k == n ? 0 : k)];
                const float2 zr = src[g * n + (k == 0 ? 0 : n - k)];   // Z[n - k]; conj taken below
                // E = (zk + conj(zr)) / 2, O = (zk - conj(zr)) / (2i)
                const float2 E = make_float2(0.5f * (zk.x + zr.x), 0.5f * (zk.y - zr.y));
                const float2 O = make_float2(0.5f * (zk.y + zr.y), -0.5f * (zk.x - zr.x));
                const float2 w = pt[k];
                float2 X = make_float2(E.x + w.x * O.x - w.y * O.y, E.y + w.x * O.y + w.y * O.x);
                if (mrow && mrow[k] == 0) X = make_float2(0.f, 0.f);
                orow[k] = X;
            }
        }
        __syncthreads();   // the next group reuses the buffers
    }
}

__global__ void mask_kernel(const float2 *__restrict__ in, long long T, int M, int B, const uint8_t *__restrict__ mask,
                            float2 *__restrict__ out) {
    const long long total = T * M * B;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long l = e / ((long long)M * B);
        const int k = (int)(e % B);
        out[e] = mask[l * B + k] ? in[e] : make_float2(0.f, 0.f);
    }
}

}  // namespace

int stft_frames(long long n_samples, int N, int hop) {
    return n_samples < N ? 0 : (int)std::min<long long>((n_samples - N) / hop + 1, 1LL << 28);
}

int check_stft_args(const float *x, int M, long long n_samples, long long ld, int N, int hop) {
    SP_CHECK(M >= 1 && M <= 64, SP_EINVAL, "stft: M must be in [1, 64]");
    SP_CHECK(N >= 4 && N <= 8192 && (N & (N - 1)) == 0, SP_ENOTIMPL, "stft: N must be a power of two in [4, 8192]");
    SP_CHECK(hop >= 1, SP_EINVAL, "stft: hop must be >= 1");
    SP_CHECK(n_samples >= 0 && ld >= n_samples, SP_EINVAL, "stft: need 0 <= n_samples <= ld");
    SP_CHECK(x || n_samples < N, SP_EINVAL, "stft: null samples pointer");
    SP_CHECK((reinterpret_cast<uintptr_t>(x) & 3) == 0, SP_EINVAL, "stft: samples must be 4-byte aligned");
    return SP_OK;
}

int launch_stft(const float *x, long long ld, int M, int N, int hop, int T, const uint8_t *mask, void *frames,
                cudaStream_t s) {
    if (T == 0) return SP_OK;
    const int n = N / 2;
    int lg_n = 0;
    while ((1 << lg_n) < n) ++lg_n;
    const int fpc = std::max(1, kStftPoints / (n * M));
    const size_t smem = (size_t)2 * fpc * M * n * sizeof(float2) + (size_t)std::max(n / 2, 1) * sizeof(float2) +
                        (size_t)(n + 1) * sizeof(float2) + (size_t)N * sizeof(float);
    SP_CHECK(smem <= 232448, SP_ENOTIMPL, "stft: transform too large for shared memory");
    if (smem > 48 * 1024) SP_TRY(ensure_max_smem((const void *)stft_kernel));
    const long long groups = ((long long)T + fpc - 1) / fpc;
    const unsigned grid = (unsigned)std::min<long long>(groups, 8LL * num_sms());
    int *status = nullptr;
    SP_TRY(device_status_ptr(&status));
    stft_kernel<<<grid, kStftThreads, smem, s>>>(x, ld, M, N, lg_n, hop, T, fpc, mask, (float2 *)frames, status);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

}  // namespace sp

using namespace sp;

extern "C" {

int sp_stft(const float *samples_dev, int M, long long n_samples, long long ld, int N, int hop,
            const uint8_t *mask_dev, void *frames_dev, int *T_out, void *stream) {
    SP_TRY(check_stft_args(samples_dev, M, n_samples, ld, N, hop));
    const int T = stft_frames(n_samples, N, hop);
    if (T_out) *T_out = T;
    if (T == 0) return SP_OK;
    SP_CHECK(frames_dev && (reinterpret_cast<uintptr_t>(frames_dev) & 7) == 0, SP_EINVAL,
             "sp_stft: frames_dev NULL or misaligned");
    return launch_stft(samples_dev, ld, M, N, hop, T, mask_dev, frames_dev, (cudaStream_t)stream);
}

int sp_apply_mask(const void *frames_dev, int T, int M, int B, const uint8_t *mask_dev, void *out_dev, void *stream) {
    SP_CHECK(T >= 0 && T <= (1 << 28) && M >= 1 && M <= 64 && B >= 1, SP_EINVAL, "sp_apply_mask: bad sizes");
    if (T == 0) return SP_OK;
    SP_CHECK(frames_dev && mask_dev && out_dev, SP_EINVAL, "sp_apply_mask: null pointer");
    SP_CHECK((reinterpret_cast<uintptr_t>(frames_dev) & 7) == 0 && (reinterpret_cast<uintptr_t>(out_dev) & 7) == 0,
             SP_EINVAL, "sp_apply_mask: frames must be 8-byte aligned");
    const long long total = (long long)T * M * B;
    const unsigned grid = (unsigned)std::min<long long>((total + 255) / 256, 8LL * num_sms());
    mask_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>((const float2 *)frames_dev, T, M, B, mask_dev,
                                                         (float2 *)out_dev);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

}  // extern "C"
