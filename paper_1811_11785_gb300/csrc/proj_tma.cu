// GEMM1 of SVD-PHAT (Eq. 3, Eq. 7, Eq. 12) for 7-microphone arrays with the STFT fed by TMA:
// Z^T = X^T conj(V) for tiles of 128 frames, the PHAT cross spectra X produced straight into
// tensor memory, V streamed from L2 into shared memory, FP32 accumulation in tensor memory.
//
// STFT staging.  The frames [T][7][B] complex64 are viewed as rows of two consecutive
// microphone rows (16 B bytes, a multiple of 16): microphone row u = 7t + m is half e = u & 1
// of row u >> 1.  For odd B (every power-of-two N) the second half starts 8 bytes off a
// 16-byte boundary, so two tensor maps cover the halves:
//   e = 0: base = frames,                 inner extent B complex,      rows ceil(7T / 2)
//   e = 1: base = frames + (B - 1) cplx,  inner extent B + 1 complex,  rows floor(7T / 2)
// A raw slot holds `cpr` chunks of 4 bins of one tile: for e = 0 the bins 4c0 .. 4c0 + 4cpr - 1
// (box of 4 cpr complex), for e = 1 one complex more on each side (box of 4 cpr + 2, starting
// at bin 4c0 - 1, the nearest 16-byte boundary).  A tile covers 448 rows (two boxes of 224).
// Everything outside the tensors (bins >= B, frames >= T, the missing second half of the last
// row when 7T is odd) reads as zero, and a zero spectrum entry is a zero cross spectrum
// (Eq. 3 with the |X|^2 < 1e-30 rule), so the producers need no bounds logic.
//
// Producers.  Twelve warps in three groups; group g takes the chunks g, g + 3, ... of the
// CTA's sequence and owns A stage g in tensor memory (96 columns: pair p, bin b of the chunk
// at column 24 b + p, (Re, Im) packed as two 16-bit values; V is stored in the same
// bin-major order, pairs 21-23 of a bin zero).  A thread is one frame (its TMEM lane): it
// copies its 7 x 4 raw values out of the raw slot (releasing the slot at once), then per bin
// normalises the 7 values, forms the 21 pairs and writes the bin's 24 columns with three
// 8-column tcgen05.st.  The group that produced a tile's last chunk then drains that tile's
// Z from tensor memory to global memory.  One warp streams raw slots by TMA, one V atoms, one
// issues the MMAs (A from tensor memory, B = V from shared memory, 12 K16 steps per chunk).
// Fifteen warps leave every thread 128 registers (a scheduler holds at most four warps).
// V arrives in three stages where shared memory allows (two for wide bases): every SM reads the
// same 2.4 MB of V in the same chunk order, and its L2 latency, not the STFT's, is the one the
// third stage hides (measured 336 -> 313 us per 65,536 frames).  Two paths of about the same
// length then bound the kernel and overlap well: the STFT slices by TMA (rows of 32-80 bytes;
// 278 us on their own, 3.4-4.2 TB/s even from L2) and the producer / MMA pipeline around
// tensor memory (298 us without any STFT load; 230 us without the MMAs as well, 214 us
// without the producers' PHAT work and tensor-memory stores instead).  Two accumulators taking
// alternate K16 steps changed nothing (315 us), so it is not the accumulation chain.
//
// Every mbarrier wait is bounded; a wait that gives up records an error in the status word
// and the CTA drains its in-flight TMA loads and MMAs before it frees tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "common.h"
#include "debug.cuh"
#include "ptx.cuh"

namespace sp {
namespace {

constexpr int kM = 7;                    // microphones
constexpr int kP = 21;                   // pairs
constexpr int kSteps = 12;               // K16 MMA steps per chunk (4 bins x 24 pair slots)
constexpr int kGroups = 3;               // producer groups = A stages in tensor memory
constexpr int kAStageCols = 96;          // TMEM columns per A stage
constexpr int kRawWarp = 12, kVWarp = 13, kMmaWarp = 14;
constexpr int kThreads = 15 * 32;
constexpr int kTileRows = 64 * kM;       // 448 rows of two microphone rows per 128 frames
constexpr int kBoxRows = kTileRows / 2;  // 224 (a box spans at most 256 rows)
constexpr int kChunkElems = 192;         // 16-bit elements of a chunk in the V layout
constexpr long long kDrainBudget = 4000000000LL;

struct Params {
    int T, B, n_chunks, n1, K, n_tiles;
    int n_raw_loads;    // raw slot loads per tile = ceil(n_chunks / CPR)
    int n_zbuf;         // Z accumulators in tensor memory (1 or 2)
    int z_cols;         // TMEM column offset of the second Z accumulator
    int a_col0;         // first A stage column
    int e0_bytes;       // bytes of the e = 0 region of a raw slot (448 rows x 32 CPR)
    int slot_bytes;     // bytes of a raw slot
    int v_stage_bytes;  // bytes of a V stage (3 atoms x n1 rows x 128)
    float inv_vscale;
    float2 *z_out;      // [T][K] complex64
    float *zn2_out;     // [T] or null
    int *status;        // device status word
    long long budget;   // SM cycles per bounded wait
};

template <int BF16>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
    if (BF16) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    } else {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
}

// pairs p = (i, j), i < j < 7, in Eq. 7 order
struct Pairs7 {
    int i[kP], j[kP];
};
constexpr Pairs7 make_pairs7() {
    Pairs7 t{};
    int n = 0;
    for (int i = 0; i < kM; ++i)
        for (int j = i + 1; j < kM; ++j) {
            t.i[n] = i;
            t.j[n] = j;
            ++n;
        }
    return t;
}

// CPR chunks per raw slot, NRAW raw slots, NV V stages (3 V stages and 3 raw slots of one chunk
// where shared memory allows, else 2 V stages)
template <int BF16, int CPR, int NRAW, int NV>
__global__ void __maxnreg__(128)
    svd_proj_tma_kernel(const __grid_constant__ CUtensorMap tmap_v, const __grid_constant__ CUtensorMap tmap_e0,
                        const __grid_constant__ CUtensorMap tmap_e1, const Params prm) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n1 = prm.n1;
    uint8_t *vbuf = smem;                                   // NV V stages
    uint8_t *rawbuf = smem + NV * prm.v_stage_bytes;        // NRAW raw slots
    uint64_t *bars = reinterpret_cast<uint64_t *>(rawbuf + NRAW * prm.slot_bytes);
    uint64_t *full_raw = bars, *empty_raw = bars + 4;       // up to 4 raw slots
    uint64_t *full_a = bars + 8, *empty_a = bars + 11;      // 3 A stages
    uint64_t *full_v = bars + 14, *empty_v = bars + 17;
    uint64_t *zfull = bars + 20, *zempty = bars + 22, *drain = bars + 24;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 25);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 26);
    const long long budget = prm.budget;

    if (tid == 0) {
        for (int i = 0; i < NRAW; ++i) {
            ptx::mbar_init(&full_raw[i], 1);
            ptx::mbar_init(&empty_raw[i], 4 * CPR);
        }
        for (int i = 0; i < kGroups; ++i) {
            ptx::mbar_init(&full_a[i], 4);
            ptx::mbar_init(&empty_a[i], 1);
        }
        for (int i = 0; i < NV; ++i) {
            ptx::mbar_init(&full_v[i], 1);
            ptx::mbar_init(&empty_v[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(&zfull[i], 1);
            ptx::mbar_init(&zempty[i], 128);
        }
        ptx::mbar_init(drain, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    if (warp == kVWarp && lane == 0) ptx::prefetch_tmap(&tmap_v);
    if (warp == kRawWarp && lane == 0) {
        ptx::prefetch_tmap(&tmap_e0);
        ptx::prefetch_tmap(&tmap_e1);
    }
    if (warp == kMmaWarp) {
        ptx::tmem_alloc(tmem_slot, 512);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int n_chunks = prm.n_chunks;
    const int my_tiles = prm.n_tiles > (int)blockIdx.x ? (prm.n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto give_up = [&]() {
        *abort_flag = 1;
        atomicOr(prm.status, 1);
    };

    if (warp < kRawWarp) {
        // -------- producers: group g, TMEM lane quarter q4, frame row f
        constexpr Pairs7 tab = make_pairs7();   // compile-time register indices below
        const int q4 = warp & 3, grp = warp >> 2;
        const int f = q4 * 32 + lane;
        constexpr int pitch0 = 32 * CPR, pitch1 = 32 * CPR + 16;
        const uint32_t raw_base = ptx::smem_u32(rawbuf);
        const uint32_t lane_addr = tmem + ((uint32_t)(q4 * 32) << 16);
        const uint32_t a_base = lane_addr + (uint32_t)(prm.a_col0 + grp * kAStageCols);
        // this group's chunks j = grp, grp + 3, ... of the CTA's sequence as (tile li, chunk c)
        int li = 0, c = grp;
        while (c >= n_chunks) {
            c -= n_chunks;
            ++li;
        }
        for (int use = 0; li < my_tiles; ++use) {
            const int h = li * prm.n_raw_loads + c / CPR;   // raw slot load of this chunk
            const int slot = h % NRAW;
            if (ptx::warp_flag(abort_flag)) break;
            if (!ptx::mbar_wait_warp(&full_raw[slot], (uint32_t)((h / NRAW) & 1), budget)) {
                if (lane == 0) give_up();
                break;
            }
            // raw values of this frame's 4 bins for every microphone, then release the slot
            float2 x[kM][4];
            const uint32_t sb = raw_base + (uint32_t)(slot * prm.slot_bytes + (c % CPR) * 32);
#pragma unroll
            for (int m = 0; m < kM; ++m) {
                // microphone row u = 7 f + m is half u & 1 of raw row u >> 1 (bin 0 of the slot's
                // first chunk at +8 in the second half, whose box starts one bin early)
                const int u = f * kM + m, r = u >> 1;
                const uint32_t mo = (u & 1) ? (uint32_t)(prm.e0_bytes + r * pitch1 + 8) : (uint32_t)(r * pitch0);
                if (!dcheck((c % CPR) * 32 + mo + 32 <= (uint32_t)prm.slot_bytes, prm.status)) {
#pragma unroll
                    for (int b = 0; b < 4; ++b) x[m][b] = make_float2(0.f, 0.f);
                    continue;
                }
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];"
                                 : "=f"(x[m][b].x), "=f"(x[m][b].y)
                                 : "r"(sb + mo + b * 8));
            }
            __syncwarp();
            if (lane == 0) {
                // the last chunk of a tile may be alone in its slot: it arrives for both
                const bool alone = CPR == 2 && c == n_chunks - 1 && (n_chunks & 1);
                ptx::mbar_arrive_cnt(&empty_raw[slot], alone ? 2u : 1u);
            }
            if (!ptx::mbar_wait_warp(&empty_a[grp], (uint32_t)((use & 1) ^ 1), budget)) {
                if (lane == 0) give_up();
                break;
            }
            ptx::tc_fence_after();
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                // PHAT normalisation (Eq. 3): x^ = X / |X|, zero where |X|^2 < 1e-30 (in place)
#pragma unroll
                for (int m = 0; m < kM; ++m) {
                    const float2 v = x[m][b];
                    const float mag2 = v.x * v.x + v.y * v.y;
                    const float r = mag2 < 1e-30f ? 0.f : rsqrtf(mag2);
                    x[m][b] = make_float2(v.x * r, v.y * r);
                }
                // cross spectra X_ij = x^_i conj(x^_j) of the bin (Eq. 3, 7): columns 24 b + p,
                // written 8 columns at a time (each store starts on a multiple of 8)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    uint32_t w[8];
#pragma unroll
                    for (int pp = 0; pp < 8; ++pp) {
                        const int p = 8 * q + pp;
                        w[pp] = 0u;
                        if (p < kP) {
                            const float2 a0 = x[tab.i[p]][b], b0 = x[tab.j[p]][b];
                            w[pp] = pack2<BF16>(a0.x * b0.x + a0.y * b0.y, a0.y * b0.x - a0.x * b0.y);
                        }
                    }
                    ptx::tmem_st8(a_base + (uint32_t)(b * 24 + 8 * q), w);
                }
            }
            ptx::tmem_wait_st();
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&full_a[grp]);
            if (c == n_chunks - 1) {
                // this group produced the tile's last chunk: drain the tile's Z (TMEM -> FP32 global)
                const int zb = prm.n_zbuf == 2 ? (li & 1) : 0;
                const uint32_t zpar = prm.n_zbuf == 2 ? ((li >> 1) & 1) : (li & 1);
                if (!ptx::mbar_wait_warp(&zfull[zb], zpar, budget)) {
                    if (lane == 0) give_up();
                    break;
                }
                ptx::tc_fence_after();
                const long long frame = (long long)((int)blockIdx.x + li * (int)gridDim.x) * 128 + f;
                const bool live = frame < prm.T;
                float2 *zo = prm.z_out + (size_t)(live ? frame : 0) * prm.K;
                float zn2 = 0.f;
                for (int c0 = 0; c0 < n1; c0 += 32) {
                    float v[32];
                    ptx::tmem_ld32(lane_addr + (uint32_t)(zb * prm.z_cols + c0), v);
                    if (live) {
#pragma unroll
                        for (int i = 0; i < 32; i += 2) {
                            const int kk = (c0 + i) >> 1;
                            if (kk < prm.K) {
                                const float2 z = make_float2(v[i] * prm.inv_vscale, v[i + 1] * prm.inv_vscale);
                                zo[kk] = z;
                                zn2 = fmaf(z.x, z.x, fmaf(z.y, z.y, zn2));
                            }
                        }
                    }
                }
                if (prm.zn2_out && live) prm.zn2_out[frame] = zn2;
                ptx::tc_fence_before();
                ptx::mbar_arrive(&zempty[zb]);
            }
            c += kGroups;
            while (c >= n_chunks) {
                c -= n_chunks;
                ++li;
            }
        }
    } else if (warp == kRawWarp) {
        // -------- raw STFT slots: CPR chunks of one tile, both halves of its 448 rows
        if (lane == 0) {
            long long issued = -1;
            const long long n_loads = (long long)my_tiles * prm.n_raw_loads;
            const int e0_box = kBoxRows * 32 * CPR, e1_box = kBoxRows * (32 * CPR + 16);
            for (long long h = 0; h < n_loads; ++h) {
                const int slot = (int)(h % NRAW);
                if (*abort_flag) break;
                if (!ptx::mbar_wait(&empty_raw[slot], (uint32_t)(((h / NRAW) & 1) ^ 1), budget)) {
                    give_up();
                    break;
                }
                const int li = (int)(h / prm.n_raw_loads), c0 = (int)(h % prm.n_raw_loads) * CPR;
                const int row0 = ((int)blockIdx.x + li * (int)gridDim.x) * kTileRows;
                uint8_t *S = rawbuf + slot * prm.slot_bytes;
                ptx::mbar_arrive_expect_tx(&full_raw[slot], (uint32_t)prm.slot_bytes);
                for (int k = 0; k < 2; ++k) {
                    ptx::tma_load_2d(S + k * e0_box, &tmap_e0, &full_raw[slot], 8 * c0, row0 + k * kBoxRows);
                    ptx::tma_load_2d(S + prm.e0_bytes + k * e1_box, &tmap_e1, &full_raw[slot], 8 * c0,
                                     row0 + k * kBoxRows);
                }
                issued = h;
            }
            for (long long h = std::max(0LL, issued - NRAW + 1); h <= issued; ++h)
                ptx::mbar_wait(&full_raw[h % NRAW], (uint32_t)((h / NRAW) & 1), kDrainBudget);
        }
        __syncwarp();
    } else if (warp == kVWarp) {
        // -------- V atoms of each chunk (3 atoms of n1 rows), NV stages
        if (lane == 0) {
            long long issued = -1;
            const long long n_stages = (long long)my_tiles * n_chunks;
            for (long long j = 0; j < n_stages; ++j) {
                const int s = (int)(j % NV);
                if (*abort_flag) break;
                if (!ptx::mbar_wait(&empty_v[s], (uint32_t)(((j / NV) & 1) ^ 1), budget)) {
                    give_up();
                    break;
                }
                const int c = (int)(j % n_chunks);
                ptx::mbar_arrive_expect_tx(&full_v[s], (uint32_t)prm.v_stage_bytes);
                uint8_t *Vs = vbuf + s * prm.v_stage_bytes;
                for (int a = 0; a < 3; ++a)
                    ptx::tma_load_2d(Vs + a * n1 * 128, &tmap_v, &full_v[s], c * kChunkElems + a * 64, 0);
                issued = j;
            }
            for (long long j = std::max(0LL, issued - NV + 1); j <= issued; ++j)
                ptx::mbar_wait(&full_v[j % NV], (uint32_t)((j / NV) & 1), kDrainBudget);
        }
        __syncwarp();
    } else {
        // -------- MMA issue: Z (+)= A[tmem] V[smem], 12 K16 steps per chunk
        if (lane == 0) {
            const uint32_t idesc = ptx::idesc_f16(128, n1, BF16);
            long long j = 0;
            for (int li = 0; li < my_tiles; ++li) {
                const int zb = prm.n_zbuf == 2 ? (li & 1) : 0;
                const uint32_t zpar = (prm.n_zbuf == 2 ? ((li >> 1) & 1) : (li & 1)) ^ 1;
                if (*abort_flag) break;
                if (!ptx::mbar_wait(&zempty[zb], zpar, budget)) {
                    give_up();
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(zb * prm.z_cols);
                bool ok = true;
                for (int c = 0; c < n_chunks; ++c, ++j) {
                    const int s = (int)(j % kGroups), v = (int)(j % NV);
                    if (*abort_flag || !ptx::mbar_wait(&full_a[s], (uint32_t)((j / kGroups) & 1), budget) ||
                        !ptx::mbar_wait(&full_v[v], (uint32_t)((j / NV) & 1), budget)) {
                        if (!*abort_flag) give_up();
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint32_t a_tmem = tmem + (uint32_t)(prm.a_col0 + s * kAStageCols);
                    const uint32_t b_base = ptx::smem_u32(vbuf + v * prm.v_stage_bytes);
                    for (int k = 0; k < kSteps; ++k) {
                        const uint32_t bo = (k >> 2) * n1 * 128 + (k & 3) * 32;
                        ptx::mma_f16_ts(d_tmem, a_tmem + (uint32_t)(k * 8), ptx::sw128_desc(b_base + bo), idesc,
                                        (c > 0 || k > 0) ? 1u : 0u);
                    }
                    ptx::mma_commit(&empty_a[s]);
                    ptx::mma_commit(&empty_v[v]);
                }
                if (!ok) break;
                ptx::mma_commit(&zfull[zb]);
            }
            ptx::mma_commit(drain);   // completes once every MMA issued above is done
            ptx::mbar_wait(drain, 0, kDrainBudget);
        }
        __syncwarp();
    }

    ptx::tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, 512);
    }
}

}  // namespace

bool proj_tma_applies(const sp_basis *b, const void *frames) {
    const TcLayout &t = b->tc;
    return b->st->M == kM && (b->st->B & 1) == 1 && (reinterpret_cast<uintptr_t>(frames) & 15) == 0 && t.n1 > 0 &&
           t.n1 <= 224 && tc_vmap_binmajor(b, 0) != nullptr;
}

int launch_svd_proj_tma(const sp_basis *b, const void *frames, int T, int prec, void *z_out, float *zn2_out,
                        cudaStream_t s, int max_ctas) {
    if (T == 0) return SP_OK;
    const sp_steering *st = b->st;
    const TcLayout &t = b->tc;
    const int B = st->B;
    // the plan: exactly 7 microphones, odd B (the 16-byte boundary falls one complex before
    // the second half of a row), 16-byte-aligned frames, 2K <= 224 (Z accumulators and three
    // A stages in 512 TMEM columns)
    const int bf = prec == SP_PREC_BF16 ? 1 : 0;
    const CUtensorMap *vmap = t.n1 > 0 ? tc_vmap_binmajor(b, bf) : nullptr;
    if (st->M != kM || (B & 1) == 0 || (reinterpret_cast<uintptr_t>(frames) & 15) != 0 || t.n1 > 224 || !vmap)
        return SP_ENOTIMPL;
    Params p;
    p.T = T;
    p.B = B;
    p.n_chunks = t.n_chunks;
    p.n1 = t.n1;
    p.K = b->K;
    p.n_tiles = (int)(((long long)T + 127) / 128);
    // tensor memory: Z accumulators at columns 0 and z_cols (128 where it fits), then the A stages
    const int zw = (t.n1 + 31) / 32 * 32;
    p.z_cols = t.n1 <= 128 ? 128 : zw;
    p.n_zbuf = p.z_cols + zw + kGroups * kAStageCols <= 512 ? 2 : 1;
    p.a_col0 = p.n_zbuf == 2 ? p.z_cols + zw : zw;
    if (p.a_col0 + kGroups * kAStageCols > 512) return SP_ENOTIMPL;
    p.v_stage_bytes = 3 * t.n1 * 128;
    // shared memory (227 KB): three V stages and three raw slots of one chunk where they fit
    // (V's L2 latency is the longer one), else two V stages with two slots of two chunks or three
    // of one chunk
    const int slot2 = kTileRows * (64 * 2 + 16), slot1 = kTileRows * (64 + 16);
    const int over = 256 + 1024;   // barriers, alignment slack
    int nv = 3, cpr = 1, n_raw = 3;
    if (3 * p.v_stage_bytes + 3 * slot1 + over > 232448) {
        nv = 2;
        if (2 * p.v_stage_bytes + 2 * slot2 + over <= 232448) {
            cpr = 2;
            n_raw = 2;
        } else if (2 * p.v_stage_bytes + 3 * slot1 + over > 232448) {
            return SP_ENOTIMPL;
        }
    }
    p.slot_bytes = cpr == 2 ? slot2 : slot1;
    p.e0_bytes = kTileRows * 32 * cpr;
    p.n_raw_loads = (p.n_chunks + cpr - 1) / cpr;
    p.inv_vscale = 1.f / b->v_scale;
    p.z_out = (float2 *)z_out;
    p.zn2_out = zn2_out;
    SP_TRY(device_status_ptr(&p.status));
    p.budget = wait_budget();
    // the two views of the frames (float32 elements; rows of two microphone rows)
    const uint64_t rows_all = ((uint64_t)T * kM + 1) / 2, rows_full = (uint64_t)T * kM / 2;
    const uint64_t pitch = (uint64_t)16 * B;
    CUtensorMap m0, m1;   // (T >= 1 gives at least 3 full rows)
    SP_TRY(encode_tmap_f32_2d(&m0, frames, 2 * (uint64_t)B, rows_all, pitch, 8 * cpr, kBoxRows));
    SP_TRY(encode_tmap_f32_2d(&m1, static_cast<const char *>(frames) + (size_t)(B - 1) * 8, 2 * (uint64_t)(B + 1),
                              rows_full, pitch, 8 * cpr + 4, kBoxRows));
    const int smem = nv * p.v_stage_bytes + n_raw * p.slot_bytes + over;
    using Kern = void (*)(CUtensorMap, CUtensorMap, CUtensorMap, Params);
    const Kern kern = nv == 3   ? (bf ? svd_proj_tma_kernel<1, 1, 3, 3> : svd_proj_tma_kernel<0, 1, 3, 3>)
                      : cpr == 2 ? (bf ? svd_proj_tma_kernel<1, 2, 2, 2> : svd_proj_tma_kernel<0, 2, 2, 2>)
                                 : (bf ? svd_proj_tma_kernel<1, 1, 3, 2> : svd_proj_tma_kernel<0, 1, 3, 2>);
    SP_TRY(ensure_max_smem((const void *)kern));
    const int grid = std::min(p.n_tiles, max_ctas > 0 ? std::min(max_ctas, num_sms()) : num_sms());
    kern<<<grid, kThreads, smem, s>>>(*vmap, m0, m1, p);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

}  // namespace sp
