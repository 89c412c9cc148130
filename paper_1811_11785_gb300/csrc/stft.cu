// The STFT front end of Section 2 and the binary time-frequency mask of the paper's conclusion.
//
// X_m^l[k] = sum_{n<N} w[n] x_m[l dN + n] exp(-2 pi i k n / N), k = 0 .. N/2, with the sine
// window w[n] = sin(pi (n + 1/2) / N).  Each transform is a real N-point DFT computed as an
// N/2-point complex FFT of z[j] = (w x)[2j] + i (w x)[2j + 1] (radix-2 Stockham in shared
// memory, natural order out), followed by X[k] = E[k] + exp(-2 pi i k / N) O[k] with
// E[k] = (Z[k] + conj(Z[N/2 - k])) / 2 and O[k] = (Z[k] - conj(Z[N/2 - k])) / (2i), the DFTs of
// the even and odd samples.  For N = 256, 512, 1024 one warp computes a transform with its
// points in registers (stft_warp_kernel, below); other N use stft_kernel: a CTA takes `fpc`
// frames x M channels at a time (persistent grid);
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

// ---------------------------------------------------------------- warp-per-transform FFT
// For N = 64 P (P = 4, 8, 16: N = 256, 512, 1024) a warp computes one (frame, channel)
// transform at a time with its n = N/2 = 32 P complex points held P per lane.  With
// z[n1 + 32 n2] (n1 = lane, n2 < P) and bins k = k2 + P (q + 8 r) (k2 < P, q < 8, r < 4):
//   stage A  a P-point DFT over n2 in registers, times W_n^(n1 k2)         -> Y[k2][n1]
//   stage B  8-point DFTs over m of Y[k2][a + 4 m] (a < 4), times W_32^(a q) -> U[k2][a][q]
//   stage C  4-point DFTs over a of U[k2][a][q]                             -> Z[k2 + P (q + 8 r)]
// (Cooley-Tukey n = 32 x P, then 32 = 4 x 8), each in-register DFT a radix-2 decimation in
// frequency whose output sits in bit-reversed order.  Stages exchange data through the warp's
// own shared-memory buffer (swizzled layouts, below), separated by __syncwarp.  Then the
// real-input post-processing and the store as in stft_kernel.  Window, W_n and the post-
// processing twiddles come from tables the CTA computes once.
constexpr int kWarpFftWarps = 8;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// Shared-memory layouts of the three exchanges, XOR-swizzled so that every warp access of
// the stages (rows of a stage's writes, columns of the next stage's reads) touches each
// 8-byte bank pair at most twice, the minimum for 32 lanes x 8 bytes:
//   Y[k2][n1] (stage A out, B in), U[k2][a][q] (B out, C in), Z[k] (C out, post-processing in)
__device__ __forceinline__ int yidx(int k2, int n1) { return k2 * 32 + (n1 ^ ((k2 & 3) << 2)); }
__device__ __forceinline__ int uidx(int k2, int a, int q) { return k2 * 32 + ((4 * q + a) ^ (5 * (k2 & 3))); }
__device__ __forceinline__ int zidx(int k) { return k ^ (((k >> 4) & 3) << 2); }

template <int S>
__device__ __forceinline__ int bitrev(int i) {
    int r = 0;
#pragma unroll
    for (int b = 1; b < S; b <<= 1) r = (r << 1) | ((i & b) ? 1 : 0);
    return r;
}

// In-place S-point DFT (S = 4, 8, 16), radix-2 decimation in frequency; v[i] ends as X[bitrev(i)].
// w[j] = exp(-2 pi i j / S), j < S / 2.
template <int S>
__device__ __forceinline__ void dft_dif(float2 (&v)[S], const float2 (&w)[S / 2]) {
#pragma unroll
    for (int h = S / 2; h >= 1; h >>= 1) {
#pragma unroll
        for (int s0 = 0; s0 < S; s0 += 2 * h) {
#pragma unroll
            for (int j = 0; j < h; ++j) {
                const float2 a = v[s0 + j], b = v[s0 + j + h];
                v[s0 + j] = make_float2(a.x + b.x, a.y + b.y);
                const float2 d = make_float2(a.x - b.x, a.y - b.y);
                const int e = j * (S / (2 * h));
                v[s0 + j + h] = e == 0 ? d : cmul(d, w[e]);
            }
        }
    }
}

template <int P>
__global__ void __launch_bounds__(32 * kWarpFftWarps, P <= 8 ? 3 : 2)
    stft_warp_kernel(const float *__restrict__ x, long long ld, int M, int hop, int T, int vec2,
                     const uint8_t *__restrict__ mask, float2 *__restrict__ out, int *status) {
    constexpr int n = 32 * P, N = 2 * n, B = n + 1;
    __shared__ float2 buf[kWarpFftWarps][n];
    __shared__ float2 wn[n];                  // exp(-2 pi i j / n)
    __shared__ float2 pt[n + 1];              // exp(-2 pi i k / N)
    __shared__ float2 win2[n];                // (w[2j], w[2j + 1])
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        float s_, c_;
        sincospif(-2.f * (float)j / (float)n, &s_, &c_);
        wn[j] = make_float2(c_, s_);
        win2[j] = make_float2(sinpif(((float)(2 * j) + 0.5f) / (float)N), sinpif(((float)(2 * j + 1) + 0.5f) / (float)N));
    }
    for (int k = threadIdx.x; k <= n; k += blockDim.x) {
        float s_, c_;
        sincospif(-2.f * (float)k / (float)N, &s_, &c_);
        pt[k] = make_float2(c_, s_);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2 *sb = buf[warp];
    // per-lane constants: the small DFTs' twiddles and stage A's W_n^(lane k2)
    float2 wP[P / 2], w8[4], w4[2], tA[P], tB[8];
#pragma unroll
    for (int j = 0; j < P / 2; ++j) wP[j] = wn[j * (n / P)];
#pragma unroll
    for (int j = 0; j < 4; ++j) w8[j] = wn[j * (n / 8)];
#pragma unroll
    for (int j = 0; j < 2; ++j) w4[j] = wn[j * (n / 4)];
#pragma unroll
    for (int k2 = 0; k2 < P; ++k2) tA[k2] = wn[(lane * k2) % n];
#pragma unroll
    for (int q = 0; q < 8; ++q) tB[q] = wn[((lane & 3) * q) * (n / 32)];   // W_32^(a q), a = lane mod 4
    const long long n_tasks = (long long)T * M;
    const long long stride = (long long)gridDim.x * kWarpFftWarps;
    // the samples of task tk (raw, unwindowed), loaded one task ahead of the transform
    auto load = [&](long long tk, float2 (&r)[P]) {
        const long long tt = tk / M;
        const int mm = (int)(tk % M);
        const float *row = x + (size_t)mm * ld + (size_t)tt * hop;
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int j = lane + 32 * q;
            r[q] = make_float2(0.f, 0.f);
            if (tk >= n_tasks || !dcheck(tt * hop + 2 * j + 1 < ld, status)) {
            } else if (vec2) {
                r[q] = __ldg(reinterpret_cast<const float2 *>(row) + j);
            } else {
                r[q] = make_float2(__ldg(row + 2 * j), __ldg(row + 2 * j + 1));
            }
        }
    };
    float2 nxt[P];
    load((long long)blockIdx.x * kWarpFftWarps + warp, nxt);
    for (long long task = (long long)blockIdx.x * kWarpFftWarps + warp; task < n_tasks; task += stride) {
        const long long t = task / M;
        const int m = (int)(task % M);
        // ---- stage A (the window applied to the prefetched samples; the next task's loads go out)
        float2 v[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const float2 wv = win2[lane + 32 * q];
            v[q] = make_float2(wv.x * nxt[q].x, wv.y * nxt[q].y);
        }
        load(task + stride, nxt);
        dft_dif<P>(v, wP);
        __syncwarp();   // the previous task's reads of the buffer are done
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const int k2 = bitrev<P>(i);
            sb[yidx(k2, lane)] = k2 == 0 ? v[i] : cmul(v[i], tA[k2]);
        }
        __syncwarp();
        // ---- stage B: tasks (k2, a), 4 P of them, P / 8 per lane (P = 4: lanes < 16)
        constexpr int NB = (4 * P + 31) / 32;
        float2 u[NB][8];
        int tb[NB];
#pragma unroll
        for (int r = 0; r < NB; ++r) {
            tb[r] = lane + 32 * r;
            const int k2 = tb[r] >> 2, a = tb[r] & 3;
#pragma unroll
            for (int mm = 0; mm < 8; ++mm) u[r][mm] = tb[r] < 4 * P ? sb[yidx(k2, a + 4 * mm)] : make_float2(0.f, 0.f);
            dft_dif<8>(u[r], w8);
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < NB; ++r) {
            if (tb[r] < 4 * P) {
                const int k2 = tb[r] >> 2, a = tb[r] & 3;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int q = bitrev<8>(i);
                    sb[uidx(k2, a, q)] = (a * q) == 0 ? u[r][i] : cmul(u[r][i], tB[q]);
                }
            }
        }
        __syncwarp();
        // ---- stage C: tasks (k2, q), 8 P of them, P / 4 per lane
        constexpr int NC = P / 4;
        float2 c4[NC][4];
#pragma unroll
        for (int r = 0; r < NC; ++r) {
            const int tc = lane + 32 * r;
#pragma unroll
            for (int a = 0; a < 4; ++a) c4[r][a] = sb[uidx(tc >> 3, a, tc & 7)];
            dft_dif<4>(c4[r], w4);
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < NC; ++r) {
            const int tc = lane + 32 * r, k2 = tc >> 3, q = tc & 7;
#pragma unroll
            for (int i = 0; i < 4; ++i) sb[zidx(k2 + P * (q + 8 * bitrev<4>(i)))] = c4[r][i];
        }
        __syncwarp();
        // ---- real-input post-processing and the store
        const uint8_t *mrow = mask ? mask + (size_t)t * B : nullptr;
        float2 *orow = out + ((size_t)t * M + m) * B;
#pragma unroll
        for (int i = 0; i <= P; ++i) {
            const int k = lane + 32 * i;
            if (k < B) {
                const float2 zk = sb[zidx(k == n ? 0 : k)];
                const float2 zr = sb[zidx(k == 0 ? 0 : n - k)];
                const float2 E = make_float2(0.5f * (zk.x + zr.x), 0.5f * (zk.y - zr.y));
                const float2 O = make_float2(0.5f * (zk.y + zr.y), -0.5f * (zk.x - zr.x));
                const float2 w = pt[k];
                float2 X = make_float2(E.x + w.x * O.x - w.y * O.y, E.y + w.x * O.y + w.y * O.x);
                if (mrow && mrow[k] == 0) X = make_float2(0.f, 0.f);
                orow[k] = X;
            }
        }
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
    if (N == 256 || N == 512 || N == 1024) {   // one warp per transform, points in registers
        int *status = nullptr;
        SP_TRY(device_status_ptr(&status));
        const int vec2 = ((reinterpret_cast<uintptr_t>(x) & 7) == 0 && (ld & 1) == 0 && (hop & 1) == 0) ? 1 : 0;
        const long long tasks = (long long)T * M;
        const unsigned grid = (unsigned)std::min<long long>((tasks + kWarpFftWarps - 1) / kWarpFftWarps,
                                                            8LL * num_sms());
        const int th = 32 * kWarpFftWarps;
        if (N == 256)
            stft_warp_kernel<4><<<grid, th, 0, s>>>(x, ld, M, hop, T, vec2, mask, (float2 *)frames, status);
        else if (N == 512)
            stft_warp_kernel<8><<<grid, th, 0, s>>>(x, ld, M, hop, T, vec2, mask, (float2 *)frames, status);
        else
            stft_warp_kernel<16><<<grid, th, 0, s>>>(x, ld, M, hop, T, vec2, mask, (float2 *)frames, status);
        SP_CUDA(cudaGetLastError());
        return SP_OK;
    }
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
