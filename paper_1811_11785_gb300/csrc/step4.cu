// Online step 4 of Algorithm 1 (Y_qbar = Re{W_qbar X}) with the STFT streamed by bulk copies.
//
// Same arithmetic as score_row_kernel (simt.cu): because tau_{q,i,j} = d_j - d_i with
// d_m = fs/c r_m . u_q, W_ij X_ij = y_i conj(y_j) with y_m[k] = x^_m[k] exp(-2 pi i k d_m / N),
// and sum_{i<j} Re{y_i conj(y_j)} = (|sum_m y_m|^2 - sum_m |y_m|^2) / 2 per bin.  |y_m|^2 is
// 1 for every microphone whose PHAT is defined and 0 for the others (Eq. 3 zero rule), so the
// second sum is a count: Y = (sum_k |sum_m y_m[k]|^2 - n_valid) / 2.
//
// Layout of the work: frames are taken in pairs (2 M B complex64 = 16 M B bytes, so every
// pair starts 16-byte aligned when the batch does); one CTA per SM walks its pairs through a
// ring of up to 8 shared-memory slots filled by one producer thread with cp.async.bulk, while
// 16 consumer warps compute in 4 teams (a team's 4 warps: frame 0 or 1 of the pair x even or
// odd 32-bin half).  Local pair j lands in slot j mod n_slots and is taken by team j mod 4,
// so with more slots than teams every team finds its next pair already loaded while the
// other slots stay in flight.  The odd last frame of an odd batch is read from global memory
// by its warps.  Every wait is bounded; a wait that gives up records status bit 4 and the CTA
// drains and returns.
#include <cuda_runtime.h>
#include <math.h>

#include "common.h"
#include "debug.cuh"
#include "ptx.cuh"

namespace sp {
namespace {

constexpr int kMaxSlots = 8;
constexpr int kTeams = 4;
constexpr int kConsumerWarps = 4 * kTeams;
constexpr int kThreads = (kConsumerWarps + 1) * 32;
constexpr float kZero2 = 1e-30f;
constexpr float kTwoPi = 6.28318530717958648f;

// -(k d / N) reduced to [-1/2, 1/2] cycles, with d / N = hi + lo (two floats): the product
// k hi is split exactly (fmaf) so that the reduction loses nothing for k < 2^24
__device__ __forceinline__ float cycles_frac(int k, float hi, float lo) {
    const float kf = (float)k;
    const float p0 = kf * hi;
    return -((p0 - rintf(p0)) + fmaf(kf, lo, fmaf(kf, hi, -p0)));
}
constexpr long long kDrainCycles = 4000000000LL;

struct Step4Params {
    const float2 *frames;
    int T, M, B, Q, n_pairs, n_slots;
    unsigned pair_bytes;   // 16 M B
    const float4 *tab;     // [Q][M]: d_m / N as float hi + lo, 64-bin step phasor (cos, sin)
    const int32_t *idx;
    float *score;
    int *status;
    long long budget;
};

template <int MMAX, bool EXACT>
__global__ void __launch_bounds__(kThreads, 1) step4_bulk_kernel(const Step4Params prm) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int M = EXACT ? MMAX : prm.M;
    const int B = prm.B;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned slot_bytes = (prm.pair_bytes + 127) / 128 * 128;
    const int n_slots = prm.n_slots;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + n_slots * slot_bytes);
    uint64_t *empty = full + kMaxSlots;
    float *part = reinterpret_cast<float *>(empty + kMaxSlots);          // [team][frame]
    volatile int *dec = reinterpret_cast<volatile int *>(part + 2 * kTeams);   // [team][frame]
    volatile int *abort_flag = dec + 2 * kTeams;
    if (threadIdx.x == 0) {
        for (int s = 0; s < n_slots; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], 4);
        }
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    __syncthreads();
    const int my_pairs = prm.n_pairs > (int)blockIdx.x ? (prm.n_pairs - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const long long budget = prm.budget;

    if (warp == kConsumerWarps) {
        // ---------------- producer: one bulk copy per pair of frames
        if (lane == 0) {
            int issued = -1;
            for (int i = 0; i < my_pairs; ++i) {
                const int s = i % n_slots;
                if (*abort_flag) break;
                if (!ptx::mbar_wait(&empty[s], ((i / n_slots) & 1) ^ 1, budget)) {
                    *abort_flag = 1;
                    atomicOr(prm.status, 4);
                    break;
                }
                const long long pair = (long long)blockIdx.x + (long long)i * gridDim.x;
                const bool whole = 2 * pair + 1 < prm.T;
                if (whole) {
                    ptx::mbar_arrive_expect_tx(&full[s], prm.pair_bytes);
                    ptx::bulk_load(smem + s * slot_bytes,
                                   reinterpret_cast<const uint8_t *>(prm.frames) + (size_t)pair * prm.pair_bytes,
                                   prm.pair_bytes, &full[s]);
                } else {
                    ptx::mbar_arrive(&full[s]);   // odd last frame: its warps read global memory
                }
                issued = i;
            }
            for (int i = issued - n_slots + 1; i <= issued; ++i)
                if (i >= 0) ptx::mbar_wait(&full[i % n_slots], (i / n_slots) & 1, kDrainCycles);
        }
        __syncwarp();
        return;
    }

    // ---------------- consumers: warp = (team, frame h of the pair, bin half g)
    const int team = warp >> 2, h = (warp >> 1) & 1, gh = warp & 1;
    const int bar_id = 1 + team * 2 + h;   // the two bin halves of frame h (64 threads)
    for (int i = team; i < my_pairs; i += kTeams) {
        const int s = i % n_slots;
        const float2 *smem_frame = reinterpret_cast<const float2 *>(smem + s * slot_bytes) + (size_t)h * M * B;
        // Both warps of a frame leave the loop together: the g = 0 warp reads the abort flag
        // before the barrier and both act on that one reading after it.
        const bool ok = ptx::mbar_wait_warp(&full[s], (i / n_slots) & 1, budget);
        if (!ok && lane == 0) {
            *abort_flag = 1;
            atomicOr(prm.status, 4);
        }
        if (gh == 0 && lane == 0) dec[team * 2 + h] = *abort_flag;
        ptx::named_bar_sync(bar_id, 64);
        if (dec[team * 2 + h]) break;
        const long long pair = (long long)blockIdx.x + (long long)i * gridDim.x;
        const long long t = 2 * pair + h;
        const bool whole = 2 * pair + 1 < prm.T;
        float acc = 0.f;
        int n_valid = 0;
        int q = -1;
        if (t < prm.T) q = prm.idx[t];
        if (q >= 0 && !dcheck(q < prm.Q, prm.status)) q = -1;
        if (q >= 0) {
            const float2 *fr = whole ? smem_frame : prm.frames + (size_t)t * M * B;
            // lane m: d_m / N (split into two floats) and the 64-bin step phasor, from the
            // per-direction table built with the steering matrix
            float my_hi = 0.f, my_lo = 0.f, my_sc = 1.f, my_ss = 0.f;
            if (lane < M) {
                const float4 e = __ldg(prm.tab + (size_t)q * M + lane);
                my_hi = e.x;
                my_lo = e.y;
                my_sc = e.z;
                my_ss = e.w;
            }
            float2 ph[MMAX], stp[MMAX];
            const int k_first = 32 * gh + lane;
#pragma unroll
            for (int m = 0; m < MMAX; ++m) {
                const float ehi = __shfl_sync(0xffffffffu, my_hi, m);
                const float elo = __shfl_sync(0xffffffffu, my_lo, m);
                stp[m] = make_float2(__shfl_sync(0xffffffffu, my_sc, m), __shfl_sync(0xffffffffu, my_ss, m));
                if (m < M) {
                    float sn, cs;
                    __sincosf(kTwoPi * cycles_frac(k_first, ehi, elo), &sn, &cs);
                    ph[m] = make_float2(cs, sn);
                }
            }
            // the last bin (B - 1 = N/2 when 64 | N/2) lane-parallel: lane m < M takes microphone
            // m, so the 64-bin loop below ends with a full warp
            const int k_end = ((B - 1) & 63) == 0 ? B - 1 : B;
            if (k_end < B && gh == 1) {
                float sr = 0.f, si = 0.f;
                if (lane < M) {
                    const float2 x = fr[(size_t)lane * B + (B - 1)];
                    const float mag2 = x.x * x.x + x.y * x.y;
                    const bool valid = mag2 >= kZero2;
                    const float r = valid ? rsqrtf(mag2) : 0.f;
                    n_valid += valid ? 1 : 0;
                    float sn, cs;
                    __sincosf(kTwoPi * cycles_frac(B - 1, my_hi, my_lo), &sn, &cs);
                    sr = (x.x * cs - x.y * sn) * r;   // x^ exp(i theta), theta = -2 pi (B-1) d / N
                    si = (x.x * sn + x.y * cs) * r;
                }
#pragma unroll
                for (int o = 1; o < MMAX; o <<= 1) {
                    sr += __shfl_xor_sync(0xffffffffu, sr, o);
                    si += __shfl_xor_sync(0xffffffffu, si, o);
                }
                if (lane == 0) acc = fmaf(sr, sr, si * si);
            }
            for (int k = k_first; k < k_end; k += 64) {
                float sr = 0.f, si = 0.f;
#pragma unroll
                for (int m = 0; m < MMAX; ++m) {
                    if (m < M) {
                        const float2 x = fr[(size_t)m * B + k];
                        const float mag2 = x.x * x.x + x.y * x.y;
                        const float2 w = ph[m];
                        const bool valid = mag2 >= kZero2;
                        const float r = valid ? rsqrtf(mag2) : 0.f;
                        n_valid += valid ? 1 : 0;
                        const float xr = x.x * r, xi = x.y * r;
                        sr += xr * w.x - xi * w.y;
                        si += xr * w.y + xi * w.x;
                        const float2 st = stp[m];
                        ph[m] = make_float2(w.x * st.x - w.y * st.y, w.x * st.y + w.y * st.x);
                    }
                }
                acc = fmaf(sr, sr, fmaf(si, si, acc));
            }
            acc = 0.5f * (acc - (float)n_valid);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        }
        // the two bin halves of frame h meet at their named barrier
        if (gh == 1 && lane == 0) part[team * 2 + h] = acc;
        ptx::named_bar_sync(bar_id, 64);
        if (gh == 0 && lane == 0 && t < prm.T)
            prm.score[t] = q < 0 ? __int_as_float(0x7fc00000) : acc + part[team * 2 + h];
        ptx::named_bar_sync(bar_id, 64);   // part[] and dec[] are reused by the next pair
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&empty[s]);
    }
}

}  // namespace

// Returns SP_ENOTIMPL when the bulk-copy plan does not apply (unaligned batch, M > 16, or a
// frame pair above 48 KB, which leaves fewer than four slots); the caller then uses
// score_row_kernel.
int launch_step4_bulk(const sp_steering *st, const void *frames, int T, const int32_t *idx, float *score,
                      cudaStream_t s) {
    if (T == 0) return SP_OK;
    const unsigned pair_bytes = 16u * (unsigned)st->M * (unsigned)st->B;
    if (st->M > 16 || (reinterpret_cast<uintptr_t>(frames) & 15) != 0 || pair_bytes > 48u * 1024u)
        return SP_ENOTIMPL;
    Step4Params p;
    p.frames = static_cast<const float2 *>(frames);
    p.T = T;
    p.M = st->M;
    p.B = st->B;
    p.Q = st->Q;
    p.n_pairs = (T + 1) / 2;
    p.pair_bytes = pair_bytes;
    const unsigned slot_bytes = (pair_bytes + 127) / 128 * 128;
    p.n_slots = (int)std::min<unsigned>(kMaxSlots, (200u * 1024u) / slot_bytes);   // 7 for M = 7, N = 512
    p.tab = st->step4_tab.as<float4>();
    p.idx = idx;
    p.score = score;
    SP_TRY(device_status_ptr(&p.status));
    p.budget = wait_budget();
    const int smem = (int)(p.n_slots * slot_bytes + 2 * kMaxSlots * 8 + 4 * kTeams * 4 + 16 + 128);
    auto kern = st->M == 7 ? step4_bulk_kernel<7, true>
                           : st->M <= 8 ? step4_bulk_kernel<8, false> : step4_bulk_kernel<16, false>;
    SP_TRY(ensure_max_smem((const void *)kern));
    const int grid = std::min(p.n_pairs, num_sms());
    kern<<<grid, kThreads, smem, s>>>(p);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

// Loads the bulk-copy step-4 kernel for this array on the current device and raises its
// shared-memory limit (what the first launch would otherwise do).
int prepare_step4(const sp_steering *st) {
    int *status = nullptr;
    SP_TRY(device_status_ptr(&status));   // the status word's address, cached per device
    if (st->M > 16) return SP_OK;
    auto kern = st->M == 7 ? step4_bulk_kernel<7, true>
                           : st->M <= 8 ? step4_bulk_kernel<8, false> : step4_bulk_kernel<16, false>;
    cudaFuncAttributes a;
    SP_CUDA(cudaFuncGetAttributes(&a, (const void *)kern));
    return ensure_max_smem((const void *)kern);
}

}  // namespace sp
