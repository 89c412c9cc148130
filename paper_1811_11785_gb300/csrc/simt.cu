// FP32 SIMT kernels of the hot path:
//   * PHAT cross spectra (Eq. 3, stacked as Eq. 7)
//   * SRP-PHAT scores Re{W X} with a fused argmax (Eq. 5, 6, 9) -- the plain FP32 reference
//     form; the same kernel scans Re{D Z} for the FP32 SVD-PHAT path (Eq. 14)
//   * the FP32 projection Z = V^H X (Eq. 12)
//   * Algorithm 1 online step 4, Y_qbar = Re{W_qbar X}
#include <cuda_runtime.h>
#include <math.h>

#include "common.h"

namespace sp {

constexpr float kZeroMag2 = 1e-30f;  // |X|^2 below this counts as a zero spectrum entry

// ------------------------------------------------------------------------- PHAT
// One thread per (frame t, bin k).  Each microphone spectrum is normalised once
// (x^ = X / |X|), then X_ij = x^_i conj(x^_j) for the pairs i < j in Eq. 7 order:
// X[t][p*B + k].  Loads and stores are coalesced along k.
__global__ void __launch_bounds__(128) phat_kernel(const float2 *__restrict__ frames, int T, int M,
                                                   int B, int nkb, float2 *__restrict__ X) {
    const long long blk = blockIdx.x;
    const long long t = blk / nkb;
    const int k = (int)(blk % nkb) * 128 + threadIdx.x;
    if (t >= T || k >= B) return;
    float2 xh[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        if (m < M) {
            const float2 v = __ldg(frames + ((size_t)t * M + m) * B + k);
            const float mag2 = v.x * v.x + v.y * v.y;
            const float r = mag2 < kZeroMag2 ? 0.f : rsqrtf(mag2);
            xh[m] = make_float2(v.x * r, v.y * r);
        }
    }
    const size_t L = (size_t)(M * (M - 1) / 2) * B;
    float2 *out = X + (size_t)t * L + k;
    int p = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
#pragma unroll
        for (int j = i + 1; j < 16; ++j) {
            if (j < M) {
                const float2 a = xh[i], b = xh[j];
                out[(size_t)p * B] = make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
                ++p;
            }
        }
    }
}

int launch_phat(const void *frames, int T, int M, int B, void *X, cudaStream_t s) {
    SP_CHECK(M >= 2 && M <= 16, SP_ENOTIMPL, "PHAT kernel supports 2..16 microphones");
    if (T == 0) return SP_OK;
    const int nkb = (B + 127) / 128;
    const long long blocks = (long long)T * nkb;
    phat_kernel<<<(unsigned)blocks, 128, 0, s>>>((const float2 *)frames, T, M, B, nkb, (float2 *)X);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

// ------------------------------------------------------------------------- argmax keys
// A score and its index packed so that a 64-bit unsigned max picks the larger score and,
// on equal scores, the lower index.  0 means "no (non-NaN) score yet".
__device__ __forceinline__ unsigned long long pack_key(float s, int q) {
    uint32_t u = __float_as_uint(s);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)u << 32) | (uint32_t)(~(uint32_t)q);
}
__device__ __forceinline__ float key_score(unsigned long long k) {
    uint32_t u = (uint32_t)(k >> 32);
    u = (u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u;
    return __uint_as_float(u);
}

__global__ void finalize_keys_kernel(const unsigned long long *__restrict__ keys, int T,
                                     const int32_t *__restrict__ remap, int32_t *__restrict__ idx,
                                     float *__restrict__ best) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const unsigned long long k = keys[t];
    const int32_t r = (int32_t)(~(uint32_t)k);
    idx[t] = k ? (remap ? remap[r] : r) : -1;
    if (best) best[t] = k ? key_score(k) : __int_as_float(0x7fc00000);
}

// ------------------------------------------------------------------------- Re{A X} + argmax
// Y[q][t] = sum_l Re(A[q][l] X[t][l]) = sum_l (Ar Xr - Ai Xi) over a contraction of Lc
// complex entries; a 128 q x 128 t tile per item, 8 x 8 outputs per thread, K step of 8
// complex entries double-buffered through shared memory.  The tile's best (score, q) per
// frame is merged across items with a 64-bit atomicMax on the packed key.
// List mode (count != null): the rows of X are list[0 .. *count), read from device memory
// when the kernel starts, and keys are indexed by list position; CTAs stride over the
// (q tile, t tile) items, so an empty list costs one read per CTA.
// Blocked summation (blocked != 0, long contractions such as SRP's 2L = 10,794 terms): each
// output's register accumulator covers one block of RA_K * kBlockIters complex entries and
// is then added to a running total in shared memory (64 KB of dynamic shared memory, one
// column per thread, conflict-free).  The partial sums that round then stay below
// 2 * 256 in magnitude instead of growing to L, so the FP32 rounding error of a score
// drops from about u L sqrt(2L) to about u L sqrt(L / 256) (u = 2^-24).
constexpr int RA_M = 128, RA_N = 128, RA_K = 8;
constexpr int kBlockIters = 32;                 // 256 complex entries per block
constexpr int kBlockedSmem = 64 * 256 * 4;      // running totals: 64 outputs x 256 threads

__global__ void __launch_bounds__(256, 2)
    re_argmax_kernel(const float2 *__restrict__ A, int Qa, int Lc, const float2 *__restrict__ X, int T_in,
                     int nq, unsigned long long *__restrict__ keys, const int32_t *__restrict__ list,
                     const int *__restrict__ count, int blocked) {
    __shared__ __align__(16) float As[2][2 * RA_K][RA_M + 4];
    __shared__ __align__(16) float Bs[2][2 * RA_K][RA_N + 4];
    extern __shared__ float tot_s[];   // [64][256] when blocked
    const int tid = threadIdx.x;
    const int T = count ? *count : T_in;
    const long long n_items = (long long)nq * (((long long)T + RA_N - 1) / RA_N);
    for (long long blk = blockIdx.x; blk < n_items; blk += gridDim.x) {
        const int q0 = (int)(blk % nq) * RA_M;
        const long long t0 = (blk / nq) * RA_N;
        const int lr = tid >> 1, lk = (tid & 1) * 4;   // load mapping: row, first complex column
        const int ty = tid >> 4, tx = tid & 15;         // compute mapping

        const bool a_ok = q0 + lr < Qa;
        const bool b_ok = t0 + lr < T;
        const float2 *arow = A + (size_t)(a_ok ? q0 + lr : 0) * Lc;
        const long long brow_i = b_ok ? (list ? (long long)list[t0 + lr] : t0 + lr) : 0;
        const float2 *brow = X + (size_t)brow_i * Lc;

        float2 ra[4], rb[4];
        auto gload = [&](int k0) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = k0 + lk + i;
                ra[i] = (a_ok && k < Lc) ? __ldg(arow + k) : make_float2(0.f, 0.f);
                rb[i] = (b_ok && k < Lc) ? __ldg(brow + k) : make_float2(0.f, 0.f);
            }
        };
        auto sstore = [&](int buf) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                As[buf][2 * (lk + i)][lr] = ra[i].x;
                As[buf][2 * (lk + i) + 1][lr] = ra[i].y;
                Bs[buf][2 * (lk + i)][lr] = rb[i].x;
                Bs[buf][2 * (lk + i) + 1][lr] = rb[i].y;
            }
        };

        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
        if (blocked)
#pragma unroll
            for (int e = 0; e < 64; ++e) tot_s[e * 256 + tid] = 0.f;

        gload(0);
        sstore(0);
        __syncthreads();
        int buf = 0, it = 0;
        for (int k0 = 0; k0 < Lc; k0 += RA_K) {
            const bool more = k0 + RA_K < Lc;
            if (more) gload(k0 + RA_K);
#pragma unroll
            for (int kk = 0; kk < RA_K; ++kk) {
                float ar[8], ai[8], br[8], bi[8];
                *(float4 *)&ar[0] = *(const float4 *)&As[buf][2 * kk][ty * 4];
                *(float4 *)&ar[4] = *(const float4 *)&As[buf][2 * kk][64 + ty * 4];
                *(float4 *)&ai[0] = *(const float4 *)&As[buf][2 * kk + 1][ty * 4];
                *(float4 *)&ai[4] = *(const float4 *)&As[buf][2 * kk + 1][64 + ty * 4];
                *(float4 *)&br[0] = *(const float4 *)&Bs[buf][2 * kk][tx * 4];
                *(float4 *)&br[4] = *(const float4 *)&Bs[buf][2 * kk][64 + tx * 4];
                *(float4 *)&bi[0] = *(const float4 *)&Bs[buf][2 * kk + 1][tx * 4];
                *(float4 *)&bi[4] = *(const float4 *)&Bs[buf][2 * kk + 1][64 + tx * 4];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        acc[i][j] = fmaf(ar[i], br[j], acc[i][j]);
                        acc[i][j] = fmaf(-ai[i], bi[j], acc[i][j]);
                    }
            }
            if (more) sstore(buf ^ 1);
            __syncthreads();
            buf ^= 1;
            if (blocked && ++it == kBlockIters) {   // close the block: total += block sum
                it = 0;
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        tot_s[(i * 8 + j) * 256 + tid] += acc[i][j];
                        acc[i][j] = 0.f;
                    }
            }
        }
        if (blocked)
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = tot_s[(i * 8 + j) * 256 + tid] + acc[i][j];

        // per-thread best over its 8 q rows (ascending q), for each of its 8 frames
        unsigned long long *red = reinterpret_cast<unsigned long long *>(&As[0][0][0]);  // [16][128]
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int tcol = (j < 4) ? tx * 4 + j : 64 + tx * 4 + (j - 4);
            unsigned long long best = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int q = q0 + ((i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4));
                const float v = acc[i][j];
                if (q < Qa && !isnan(v)) {
                    const unsigned long long key = pack_key(v, q);
                    best = key > best ? key : best;
                }
            }
            red[ty * RA_N + tcol] = best;
        }
        __syncthreads();
        if (tid < RA_N) {
            unsigned long long best = 0;
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                const unsigned long long k = red[r * RA_N + tid];
                best = k > best ? k : best;
            }
            const long long t = t0 + tid;
            if (t < T && best) atomicMax(keys + t, best);
        }
        __syncthreads();   // the next item reuses the shared tiles
    }
}

// List mode's results: frame list[r] gets the argmax (through remap) and score of keys[r].
__global__ void finalize_list_kernel(const unsigned long long *__restrict__ keys, const int *__restrict__ count,
                                     const int32_t *__restrict__ list, const int32_t *__restrict__ remap,
                                     int32_t *__restrict__ idx, float *__restrict__ best) {
    const int n = *count;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const unsigned long long k = keys[r];
        const int t = list[r];
        const int32_t q = (int32_t)(~(uint32_t)k);
        idx[t] = k ? (remap ? remap[q] : q) : -1;
        if (best) best[t] = k ? key_score(k) : __int_as_float(0x7fc00000);
    }
}

static int launch_re_argmax(const void *A, int Qa, int Lc, const void *X, int T, uint64_t *keys,
                            const int32_t *remap, int32_t *idx, float *best, cudaStream_t s) {
    if (T == 0) return SP_OK;
    SP_CUDA(cudaMemsetAsync(keys, 0, (size_t)T * 8, s));
    const int nq = (Qa + RA_M - 1) / RA_M;
    const long long nt = ((long long)T + RA_N - 1) / RA_N;
    const int blocked = Lc > RA_K * kBlockIters ? 1 : 0;
    if (blocked) SP_TRY(ensure_max_smem((const void *)re_argmax_kernel));
    re_argmax_kernel<<<(unsigned)(nq * nt), 256, blocked ? kBlockedSmem : 0, s>>>(
        (const float2 *)A, Qa, Lc, (const float2 *)X, T, nq, (unsigned long long *)keys, nullptr, nullptr, blocked);
    SP_CUDA(cudaGetLastError());
    finalize_keys_kernel<<<(T + 255) / 256, 256, 0, s>>>((const unsigned long long *)keys, T, remap, idx, best);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

int launch_srp_argmax(const void *A, int Qa, int Lc, const void *X, int T, uint64_t *keys,
                      int32_t *idx, float *best, cudaStream_t s) {
    return launch_re_argmax(A, Qa, Lc, X, T, keys, nullptr, idx, best, s);
}

// FP32 exhaustive scan Re{D Z} (Eq. 14) over the class representatives only.
// The same FP32 scan for the frames list[0 .. *count) of Z (count on the device, at most
// T_cap); keys[0 .. *count) must be zero.  Writes idx / best of the listed frames only.
int launch_svd_scan_f32_list(const sp_basis *b, const void *Z, int T_cap, const int *count, const int32_t *list,
                             uint64_t *keys, int32_t *idx, float *best, cudaStream_t s) {
    if (T_cap == 0) return SP_OK;
    const int Qa = (int)b->st->reps.size();
    const int nq = (Qa + RA_M - 1) / RA_M;
    const long long items = (long long)nq * (((long long)T_cap + RA_N - 1) / RA_N);
    const unsigned grid = (unsigned)std::min<long long>(items, 2LL * num_sms());
    re_argmax_kernel<<<grid, 256, 0, s>>>(b->Dc32r.as<float2>(), Qa, b->K, (const float2 *)Z, T_cap, nq,
                                          (unsigned long long *)keys, list, count, 0);
    SP_CUDA(cudaGetLastError());
    const unsigned fgrid = (unsigned)std::min<long long>(((long long)T_cap + 255) / 256, num_sms());
    finalize_list_kernel<<<fgrid, 256, 0, s>>>((const unsigned long long *)keys, count, list,
                                               b->st->d_reps.as<int32_t>(), idx, best);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

int launch_svd_scan_f32(const sp_basis *b, const void *Z, int T, uint64_t *keys, int32_t *idx,
                        float *best, cudaStream_t s) {
    return launch_re_argmax(b->Dc32r.p, (int)b->st->reps.size(), b->K, Z, T, keys, b->st->d_reps.as<int32_t>(),
                            idx, best, s);
}

// ------------------------------------------------------------------------- Z = V^H X (FP32)
// Z[t][c] = sum_l X[t][l] conj(Vt[c][l]) with Vt = V^T ([K][L] complex64).  64 t x 64 c
// tile per CTA, 4 x 4 complex outputs per thread, K step of 16 complex entries.
constexpr int PJ_M = 64, PJ_N = 64, PJ_K = 16;

__global__ void __launch_bounds__(256)
    project_f32_kernel(const float2 *__restrict__ X, int T, int Lc, const float2 *__restrict__ Vt, int K,
                       int nk, float2 *__restrict__ Z) {
    __shared__ __align__(16) float Xs[2 * PJ_K][PJ_M + 4];
    __shared__ __align__(16) float Vs[2 * PJ_K][PJ_N + 4];
    const int tid = threadIdx.x;
    const long long blk = blockIdx.x;
    const int c0 = (int)(blk % nk) * PJ_N;
    const long long t0 = (blk / nk) * PJ_M;
    const int lr = tid >> 2, lk = (tid & 3) * 4;
    const int ty = tid >> 4, tx = tid & 15;
    const bool x_ok = t0 + lr < T, v_ok = c0 + lr < K;
    const float2 *xrow = X + (size_t)(x_ok ? t0 + lr : 0) * Lc;
    const float2 *vrow = Vt + (size_t)(v_ok ? c0 + lr : 0) * Lc;
    float zr[4][4], zi[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) zr[i][j] = zi[i][j] = 0.f;
    for (int k0 = 0; k0 < Lc; k0 += PJ_K) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int k = k0 + lk + i;
            const float2 xv = (x_ok && k < Lc) ? __ldg(xrow + k) : make_float2(0.f, 0.f);
            const float2 vv = (v_ok && k < Lc) ? __ldg(vrow + k) : make_float2(0.f, 0.f);
            Xs[2 * (lk + i)][lr] = xv.x;
            Xs[2 * (lk + i) + 1][lr] = xv.y;
            Vs[2 * (lk + i)][lr] = vv.x;
            Vs[2 * (lk + i) + 1][lr] = vv.y;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < PJ_K; ++kk) {
            float xr[4], xi[4], vr[4], vi[4];
            *(float4 *)xr = *(const float4 *)&Xs[2 * kk][ty * 4];
            *(float4 *)xi = *(const float4 *)&Xs[2 * kk + 1][ty * 4];
            *(float4 *)vr = *(const float4 *)&Vs[2 * kk][tx * 4];
            *(float4 *)vi = *(const float4 *)&Vs[2 * kk + 1][tx * 4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // (xr + i xi)(vr - i vi)
                    zr[i][j] = fmaf(xr[i], vr[j], zr[i][j]);
                    zr[i][j] = fmaf(xi[i], vi[j], zr[i][j]);
                    zi[i][j] = fmaf(xi[i], vr[j], zi[i][j]);
                    zi[i][j] = fmaf(-xr[i], vi[j], zi[i][j]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const long long t = t0 + ty * 4 + i;
        if (t >= T) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = c0 + tx * 4 + j;
            if (c < K) Z[(size_t)t * K + c] = make_float2(zr[i][j], zi[i][j]);
        }
    }
}

int launch_project_f32(const sp_basis *b, const void *X, int T, void *Z, cudaStream_t s) {
    if (T == 0) return SP_OK;
    const int nk = (b->K + PJ_N - 1) / PJ_N;
    const long long nt = ((long long)T + PJ_M - 1) / PJ_M;
    project_f32_kernel<<<(unsigned)(nk * nt), 256, 0, s>>>((const float2 *)X, T, b->st->L,
                                                            (const float2 *)b->Vc32.p, b->K, nk,
                                                            (float2 *)Z);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

// ------------------------------------------------------------------------- online step 4
// Y_qbar = Re{W_qbar X} (Algorithm 1, online step 4).  Because tau_{q,i,j} = d_j - d_i with
// d_m = fs/c r_m . u_q (Eq. 2; -fs/c ||s_q - r_m|| for Eq. 1), every term factors as
// W_ij X_ij = y_i conj(y_j) with y_m[k] = x^_m[k] exp(-2 pi i k d_m / N), so
//     sum_{i<j} Re{y_i conj(y_j)} = (|sum_m y_m|^2 - sum_m |y_m|^2) / 2
// per bin: O(M) work per bin instead of O(P).  One warp per frame, lane l takes bins
// l, l + 32, ...; the phasor of mic m at bin k is advanced by exp(-2 pi i 32 d_m / N) from
// one bin of the lane to the next.  Lane m reads d_m / N (two floats, from FP64, so that
// k d_m / N is exact to ~1e-9 turns) from the per-direction table built with the steering
// matrix, forms the 32-bin step phasor and broadcasts both.
// MMAX: bound on the microphone count (EXACT: M == MMAX at compile time).
template <int MMAX, bool EXACT>
__global__ void __launch_bounds__(256)
    score_row_kernel(const float2 *__restrict__ frames, int T, int M_rt, int B, const float4 *__restrict__ tab,
                     const int32_t *__restrict__ idx, float *__restrict__ score) {
    const int M = EXACT ? MMAX : M_rt;
    const int lane = threadIdx.x & 31;
    const long long t = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (t >= T) return;
    const int q = idx[t];
    if (q < 0) {
        if (lane == 0) score[t] = __int_as_float(0x7fc00000);
        return;
    }
    float my_hi = 0.f, my_lo = 0.f, my_sc = 1.f, my_ss = 0.f;
    if (lane < M) {
        const float4 e = __ldg(tab + (size_t)q * M + lane);
        my_hi = e.x;
        my_lo = e.y;
        const float p1 = 32.f * my_hi;
        const float r1 = (p1 - rintf(p1)) + 32.f * my_lo;
        sincospif(-2.f * r1, &my_ss, &my_sc);
    }
    const float2 *fr = frames + (size_t)t * M * B;
    float2 ph[MMAX], stp[MMAX];
#pragma unroll
    for (int m = 0; m < MMAX; ++m) {
        const float ehi = __shfl_sync(0xffffffffu, my_hi, m);
        const float elo = __shfl_sync(0xffffffffu, my_lo, m);
        stp[m] = make_float2(__shfl_sync(0xffffffffu, my_sc, m), __shfl_sync(0xffffffffu, my_ss, m));
        if (m < M) {
            const float kf = (float)lane;
            const float p0 = kf * ehi;
            const float r0 = (p0 - rintf(p0)) + fmaf(kf, elo, fmaf(kf, ehi, -p0));
            float s, c;
            sincospif(-2.f * r0, &s, &c);
            ph[m] = make_float2(c, s);
        }
    }
    float acc = 0.f;
    // three bins per lane per round: 3 * M independent loads in flight
    for (int k0 = lane; k0 < B; k0 += 96) {
        float2 v[3][MMAX];
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
            for (int m = 0; m < MMAX; ++m)
                v[u][m] = (m < M && k0 + 32 * u < B) ? __ldg(fr + (size_t)m * B + k0 + 32 * u) : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            float sr = 0.f, si = 0.f, en = 0.f;
#pragma unroll
            for (int m = 0; m < MMAX; ++m) {
                if (m < M) {
                    const float2 x = v[u][m];
                    const float mag2 = x.x * x.x + x.y * x.y;
                    const float2 w = ph[m];
                    const float r = mag2 >= kZeroMag2 ? rsqrtf(mag2) : 0.f;
                    const float xr = x.x * r, xi = x.y * r;
                    const float yr = xr * w.x - xi * w.y, yi = xr * w.y + xi * w.x;
                    sr += yr;
                    si += yi;
                    en += yr * yr + yi * yi;
                    const float2 st = stp[m];
                    ph[m] = make_float2(w.x * st.x - w.y * st.y, w.x * st.y + w.y * st.x);
                }
            }
            if (k0 + 32 * u < B) acc += 0.5f * (sr * sr + si * si - en);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) score[t] = acc;
}

int launch_score_row(const sp_steering *st, const void *frames, int T, const int32_t *idx,
                     float *score, cudaStream_t s) {
    if (T == 0) return SP_OK;
    SP_CHECK(st->M <= 16, SP_ENOTIMPL, "online step 4 supports M <= 16");
    {   // bulk-copy version where it applies (16-byte aligned batch, frame pairs <= 48 KB)
        const int rc = launch_step4_bulk(st, frames, T, idx, score, s);
        if (rc != SP_ENOTIMPL) return rc;
    }
    const long long blocks = ((long long)T + 7) / 8;
    auto kern = st->M == 7 ? score_row_kernel<7, true> : st->M <= 8 ? score_row_kernel<8, false> : score_row_kernel<16, false>;
    kern<<<(unsigned)blocks, 256, 0, s>>>((const float2 *)frames, T, st->M, st->B, st->step4_tab.as<float4>(), idx,
                                          score);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

// Loads the list-scan kernels and the warp-per-frame step-4 kernel for this array on the
// current device (what their first launches would otherwise do).
int prepare_simt(const sp_steering *st) {
    cudaFuncAttributes a;
    SP_CUDA(cudaFuncGetAttributes(&a, (const void *)re_argmax_kernel));
    SP_CUDA(cudaFuncGetAttributes(&a, (const void *)finalize_list_kernel));
    if (st->M <= 16) {
        auto kern = st->M == 7 ? score_row_kernel<7, true> : st->M <= 8 ? score_row_kernel<8, false> : score_row_kernel<16, false>;
        SP_CUDA(cudaFuncGetAttributes(&a, (const void *)kern));
    }
    return SP_OK;
}

}  // namespace sp
