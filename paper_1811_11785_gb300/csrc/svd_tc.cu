// Tensor-core SVD-PHAT on sm_103a: online steps 1-3 of Algorithm 1 in two kernels.
//
// svd_proj_kernel (persistent, one CTA per SM) -- Eq. 3, Eq. 7, Eq. 12:
//   Z^T = X^T conj(V) as a real GEMM over 2L with M = 128 frames per tile, N = 2K
//   (Re Z_k, Im Z_k interleaved), FP16 or BF16 operands, FP32 accumulator in TMEM.  The A
//   operand (the PHAT cross spectra) is produced straight into shared memory by 16 producer
//   warps (one thread per frame and bin) from the STFT frames, so X never reaches global
//   memory; V (scaled by sqrt(L))
//   streams from L2 by TMA.  Four epilogue warps drain each finished tile's Z from TMEM
//   (double-buffered) to global memory as FP32 while the producers stream the next tile.
//
// svd_scan_kernel -- Eq. 13, Eq. 14 and the rescoring:
//   Y = Re{D Z} = [Re D, -Im D] . [Re Z, Im Z] over tiles of 64 direction classes, FP16/BF16
//   operands (Z rounded from FP32), FP32 in TMEM; Y never leaves the chip.  Every scan score
//   differs from its FP32 rescoring by at most e = 2.1 u sqrt(L) ||Z|| (u: unit roundoff of
//   the operand type; sum_k |D_qk||Z_k| <= ||D_q|| ||Z|| and ||D_q|| <= ||W_q|| = sqrt(L)),
//   so the FP32 winner scores at least m - 2e in the scan, m the frame's scan maximum.  One
//   pass over the class tiles keeps a running maximum and every class at or above it minus
//   2e + 2e-6 L (at most 14 per frame; a frame with more is rescored against every class);
//   all kept classes are rescored in FP32 against FP32 Z and FP32 D, and the best (ties ->
//   lowest direction index) is the frame's direction.  The result equals an FP32 scan of
//   the same Z.  An optional device-side frame list restricts the scan to listed frames.
//
// K-dimension layout of GEMM1 (a permutation of the paper's column order p*B + k): the
// contraction is cut into stages (bin chunk c of 4 bins, pair group g of <= 24 pairs);
// in a stage, pair p (local index) and bin b sit at elements p*8 + 2b (real) and
// p*8 + 2b + 1 (imaginary), so one K16 MMA step covers 2 pairs x 4 bins and a 64-element
// 128-byte-swizzled atom covers 8 pairs.
//
// Every mbarrier wait is bounded; a wait that gives up records an error in g_status and
// the CTA drains its in-flight TMA loads and MMAs (with a fixed generous bound) before it
// frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "common.h"
#include "debug.cuh"
#include "ptx.cuh"

namespace sp {

__device__ int g_status = 0;
__device__ long long g_wait_budget = 2000000000LL;  // SM cycles per bounded wait
constexpr long long kDrainBudget = 4000000000LL;     // draining in-flight async work

static long long h_wait_budget = 2000000000LL;
long long wait_budget() { return h_wait_budget; }

// Device address of the status word, for kernels of other translation units (looked up
// once per device).
int device_status_ptr(int **out) {
    static int *cache[64] = {};
    static std::mutex mu;
    int dev = 0;
    SP_CUDA(cudaGetDevice(&dev));
    SP_CHECK(dev >= 0 && dev < 64, SP_ENOTIMPL, "device index out of range");
    std::lock_guard<std::mutex> lock(mu);
    if (!cache[dev]) {
        void *p = nullptr;
        SP_CUDA(cudaGetSymbolAddress(&p, g_status));
        cache[dev] = static_cast<int *>(p);
    }
    *out = cache[dev];
    return SP_OK;
}

int read_and_clear_device_status(cudaStream_t s, int *status) {
    int v = 0, zero = 0;
    SP_CUDA(cudaStreamSynchronize(s));
    SP_CUDA(cudaMemcpyFromSymbol(&v, g_status, sizeof(int)));
    SP_CUDA(cudaMemcpyToSymbol(g_status, &zero, sizeof(int)));
    *status = v;
    return SP_OK;
}

constexpr int kGroupPairs = 24;       // pairs per stage group (3 atoms)
constexpr int kAtomElems = 64;        // 16-bit elements per swizzle atom row
constexpr int kAtomBytes = 128 * 128; // one 128-row atom
constexpr int kGroupElems = 3 * kAtomElems;
constexpr int kMaxN1 = 288;           // GEMM1 N limit: two MMAs of N <= 256 above 256, and two V
                                      // stages of 3 atoms x n1 rows (2 x 3 x 128 n1 B) in 216 KB
constexpr int kMaxN1Smem = 144;       // widest basis of the shared-memory A plan
constexpr int kProdWarps = 16;
constexpr int kProjThreads = 22 * 32; // 16 producer, 4 epilogue, 1 TMA, 1 MMA warps
constexpr int kEpiWarp0 = 16, kTmaWarp = 20, kMmaWarp = 21;
constexpr int kZBuf = 256;            // TMEM column offset of the second Z buffer
constexpr int kScanThreads = 320;     // 8 epilogue (2 per TMEM lane quadrant), 1 TMA, 1 MMA warps
constexpr int kScanEpiWarps = 8, kScanTmaWarp = 8, kScanMmaWarp = 9;
constexpr int kN2 = 64;               // direction classes per GEMM2 tile
constexpr int kCap = 14;              // candidates kept per frame (two CTAs per SM at 2K <= 128)
constexpr int kCapH = kCap / 2;       // per half tile (a frame's two epilogue threads)
constexpr int kRingMax = 4;           // GEMM2 D-tile / TMEM buffers in flight (2 when 2K > 256)

TcLayout make_tc_layout(int P, int B, int K) {
    TcLayout t;
    t.P = P;
    t.Pp = (P + 1) / 2 * 2;
    t.steps_per_chunk = 0;
    t.atoms_per_chunk = 3;
    t.n_chunks = (B + kChunkBins - 1) / kChunkBins;
    const int G = (P + kGroupPairs - 1) / kGroupPairs;
    t.row_elems = t.n_chunks * G * kGroupElems;
    t.n1 = (2 * K + 15) / 16 * 16;
    t.k2 = (2 * K + 15) / 16 * 16;
    t.k2_atoms = (t.k2 + kAtomElems - 1) / kAtomElems;
    t.n2 = kN2;
    return t;
}

// The pairs (i, j), i < j < MMAX, in Eq. 7 order; unrolled loops over this table keep
// every x^_m access a compile-time register index.
template <int MMAX>
struct PairTab {
    int i[MMAX * (MMAX - 1) / 2];
    int j[MMAX * (MMAX - 1) / 2];
};
template <int MMAX>
constexpr PairTab<MMAX> make_pair_tab() {
    PairTab<MMAX> t{};
    int n = 0;
    for (int i = 0; i < MMAX; ++i)
        for (int j = i + 1; j < MMAX; ++j) {
            t.i[n] = i;
            t.j[n] = j;
            ++n;
        }
    return t;
}

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

__device__ __forceinline__ float2 ld_stream(const float2 *p) {
    float2 v;
    asm volatile("ld.global.nc.L2::256B.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}

// ===================================================================== GEMM1 kernel
struct ProjParams {
    const float2 *frames;
    int T, M, B, P, G, n_chunks;
    int n1, K, n_tiles;
    int n_zbuf, z_cols, a_col0, n_aslot, n_vslot;   // tensor-memory plan of svd_proj_tm_kernel
    int v_box;                                      // rows per TMA box of a V atom
    float inv_vscale;
    float2 *z_out;       // [T][K] complex64
    float *zn2_out;      // [T] ||Z||^2 or null
};

// MMAX: bound on the microphone count (EXACT: M == MMAX, known at compile time);
// DEPTH: how many items of raw STFT values are held in registers ahead of use.
template <int BF16, int MMAX, bool EXACT, int DEPTH>
__global__ void __launch_bounds__(kProjThreads, 1)
    svd_proj_kernel(const __grid_constant__ CUtensorMap tmap_v, const ProjParams prm) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n1 = prm.n1;
    const int a_stage = 3 * kAtomBytes, b_stage = 3 * n1 * 128;
    const int off_b = 2 * a_stage;
    const int off_bar = off_b + 2 * b_stage;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + off_bar);
    uint64_t *full_a = bars + 0, *full_b = bars + 2, *empty = bars + 4;
    uint64_t *zfull = bars + 6, *zempty = bars + 8, *drain = bars + 10;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 11);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 12);
    const long long budget = g_wait_budget;

    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(&full_a[i], kProdWarps);
            ptx::mbar_init(&full_b[i], 1);
            ptx::mbar_init(&empty[i], 1);
            ptx::mbar_init(&zfull[i], 1);
            ptx::mbar_init(&zempty[i], 128);
        }
        ptx::mbar_init(drain, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    if (warp == kTmaWarp && lane == 0) ptx::prefetch_tmap(&tmap_v);
    if (warp == kMmaWarp) {
        ptx::tmem_alloc(tmem_slot, 512);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int stages_per_tile = prm.n_chunks * prm.G;
    const int my_tiles = prm.n_tiles > (int)blockIdx.x ? (prm.n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto give_up = [&]() {
        *abort_flag = 1;
        atomicOr(&g_status, 1);
    };

    if (warp < kProdWarps) {
        // -------- producers: PHAT of (frame f, bin b) of every chunk of every tile.
        // The STFT stream of this CTA is a flat sequence of items (local tile, chunk); the
        // raw values of item j + DEPTH are in flight while item j is normalised and written.
        // With EXACT, the pair layout (P, groups, slots) is known at compile time.
        constexpr int NPAIR = MMAX * (MMAX - 1) / 2;
        constexpr PairTab<MMAX> tab = make_pair_tab<MMAX>();
        const int M = EXACT ? MMAX : prm.M;
        const int P = EXACT ? NPAIR : prm.P;
        const int G = EXACT ? (NPAIR + kGroupPairs - 1) / kGroupPairs : prm.G;
        const int f = tid >> 2, b = tid & 3;
        const int n_chunks = prm.n_chunks;
        const size_t frame_elems = (size_t)M * prm.B;
        // swizzled byte offset of this thread's 4 bytes in 16-byte chunk x of an atom row
        uint32_t sw[8];
#pragma unroll
        for (int x = 0; x < 8; ++x) sw[x] = f * 128 + b * 4 + ((x ^ (f & 7)) << 4);
        // load cursor: item (li, c), frame pointer, liveness
        int ld_li = 0, ld_c = 0;
        const float2 *ld_fr = prm.frames;
        bool ld_live = false;
        auto ld_seek_tile = [&]() {
            const long long frame = (long long)((int)blockIdx.x + ld_li * (int)gridDim.x) * 128 + f;
            ld_live = ld_li < my_tiles && frame < prm.T;
            ld_fr = prm.frames + (ld_live ? (size_t)frame * frame_elems : 0);
        };
        float2 raw[DEPTH][MMAX];
        auto load_next = [&](float2 (&dst)[MMAX]) {
            const int k = ld_c * kChunkBins + b;
            const bool ok = ld_live && k < prm.B;
#pragma unroll
            for (int m = 0; m < MMAX; ++m)
                dst[m] = (ok && m < M) ? ld_stream(ld_fr + (size_t)m * prm.B + k) : make_float2(0.f, 0.f);
            if (++ld_c == n_chunks) {
                ld_c = 0;
                ++ld_li;
                ld_seek_tile();
            }
        };
        ld_seek_tile();
        const int n_items = my_tiles * n_chunks;
        int st = 0;  // stage counter
        // one item: normalise the raw values, start loading a later item into the same
        // registers, then write every pair of every stage group of the item
        auto step = [&](float2 (&cur)[MMAX]) -> bool {
            float2 xh[MMAX];
#pragma unroll
            for (int m = 0; m < MMAX; ++m) {
                const float2 v = cur[m];
                const float mag2 = v.x * v.x + v.y * v.y;
                const float r = mag2 < 1e-30f ? 0.f : rsqrtf(mag2);
                xh[m] = make_float2(v.x * r, v.y * r);
            }
            load_next(cur);
            for (int g = 0; g < G; ++g, ++st) {
                const int s = st & 1;
                const uint32_t par = ((st >> 1) & 1) ^ 1;
                if (*abort_flag) return false;
                if (!ptx::mbar_wait(&empty[s], par, budget)) {
                    give_up();
                    return false;
                }
                const uint32_t A = ptx::smem_u32(smem + s * a_stage);
                uint32_t ad[8];
#pragma unroll
                for (int x = 0; x < 8; ++x) ad[x] = A + sw[x];
                // address of local pair pl: a table lookup when pl is known at compile time,
                // else the swizzle arithmetic (a runtime index would put ad[] in local memory)
                auto pair_addr = [&](int pl) -> uint32_t {
                    return (EXACT ? ad[pl & 7] : A + (uint32_t)(f * 128 + b * 4 + (((pl & 7) ^ (f & 7)) << 4))) +
                           (uint32_t)((pl >> 3) * kAtomBytes);
                };
                const int p_lo = g * kGroupPairs;
                const int npg = min(kGroupPairs, P - p_lo);
#pragma unroll
                for (int pp = 0; pp < NPAIR; ++pp) {
                    const int i = tab.i[pp], jj = tab.j[pp];
                    if (jj < M) {
                        const int p = i * M - ((i * (i + 1)) >> 1) + (jj - i - 1);
                        const int pl = p - p_lo;
                        if (pl >= 0 && pl < npg) {
                            const float2 a0 = xh[i], b0 = xh[jj];
                            const uint32_t w = pack2<BF16>(a0.x * b0.x + a0.y * b0.y, a0.y * b0.x - a0.x * b0.y);
                            asm volatile("st.shared.b32 [%0], %1;" ::"r"(pair_addr(pl)), "r"(w) : "memory");
                        }
                    }
                }
                if (npg & 1)  // zero partner slot of an odd last pair
                    asm volatile("st.shared.b32 [%0], %1;" ::"r"(pair_addr(npg)), "r"(0u) : "memory");
                ptx::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&full_a[s]);
            }
            return true;
        };
#pragma unroll
        for (int d = 0; d < DEPTH; ++d) load_next(raw[d]);
        bool ok = true;
        for (int j = 0; j < n_items && ok; j += DEPTH) {
#pragma unroll
            for (int d = 0; d < DEPTH; ++d)
                if (ok && j + d < n_items) ok = step(raw[d]);
        }
    } else if (warp < kEpiWarp0 + 4) {
        // -------- epilogue: Z of each finished tile, TMEM -> FP32 global
        const int q4 = warp - kEpiWarp0;   // TMEM lane quarter of this warp
        const int r = q4 * 32 + lane;      // frame row within the tile
        for (int li = 0; li < my_tiles; ++li) {
            const int zb = li & 1;
            if (ptx::warp_flag(abort_flag)) break;
            if (!ptx::mbar_wait_warp(&zfull[zb], (li >> 1) & 1, budget)) {
                if (lane == 0) give_up();
                break;
            }
            ptx::tc_fence_after();
            const long long frame = (long long)((int)blockIdx.x + li * (int)gridDim.x) * 128 + r;
            const bool live = frame < prm.T;
            float2 *zo = prm.z_out + (size_t)(live ? frame : 0) * prm.K;
            float zn2 = 0.f;
            for (int c0 = 0; c0 < n1; c0 += 32) {
                float v[32];
                ptx::tmem_ld32(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(zb * kZBuf + c0), v);
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
    } else if (warp == kTmaWarp) {
        if (lane == 0) {
            int issued = -1;
            const int n_stages = my_tiles * stages_per_tile;
            for (int st = 0; st < n_stages; ++st) {
                const int s = st & 1;
                if (*abort_flag) break;
                if (!ptx::mbar_wait(&empty[s], ((st >> 1) & 1) ^ 1, budget)) {
                    give_up();
                    break;
                }
                const int sl = st % stages_per_tile;
                const int g = sl % prm.G;
                const int npg = min(kGroupPairs, prm.P - g * kGroupPairs);
                const int atoms = (((npg + 1) >> 1) + 3) >> 2;
                ptx::mbar_arrive_expect_tx(&full_b[s], (uint32_t)(atoms * n1 * 128));
                uint8_t *Bs = smem + off_b + s * b_stage;
                for (int a = 0; a < atoms; ++a)
                    ptx::tma_load_2d(Bs + a * n1 * 128, &tmap_v, &full_b[s], sl * kGroupElems + a * kAtomElems, 0);
                issued = st;
            }
            for (int st = max(0, issued - 1); st <= issued; ++st)
                ptx::mbar_wait(&full_b[st & 1], (st >> 1) & 1, kDrainBudget);
        }
        __syncwarp();
    } else {  // kMmaWarp
        if (lane == 0) {
            const uint32_t idesc = ptx::idesc_f16(128, n1, BF16);
            int st = 0;
            for (int li = 0; li < my_tiles; ++li) {
                const int zb = li & 1;
                if (*abort_flag) break;
                if (!ptx::mbar_wait(&zempty[zb], ((li >> 1) & 1) ^ 1, budget)) {
                    give_up();
                    break;
                }
                ptx::tc_fence_after();
                bool ok = true;
                for (int sl = 0; sl < stages_per_tile; ++sl, ++st) {
                    const int s = st & 1;
                    const uint32_t par = (st >> 1) & 1;
                    if (*abort_flag || !ptx::mbar_wait(&full_a[s], par, budget) ||
                        !ptx::mbar_wait(&full_b[s], par, budget)) {
                        if (!*abort_flag) give_up();
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const int g = sl % prm.G;
                    const int npg = min(kGroupPairs, prm.P - g * kGroupPairs);
                    const int steps = (npg + 1) >> 1;
                    const uint32_t a_base = ptx::smem_u32(smem + s * a_stage);
                    const uint32_t b_base = ptx::smem_u32(smem + off_b + s * b_stage);
                    for (int k = 0; k < steps; ++k) {
                        const uint32_t ao = (k >> 2) * kAtomBytes + (k & 3) * 32;
                        const uint32_t bo = (k >> 2) * n1 * 128 + (k & 3) * 32;
                        ptx::mma_f16(tmem + zb * kZBuf, ptx::sw128_desc(a_base + ao), ptx::sw128_desc(b_base + bo),
                                     idesc, (sl > 0 || k > 0) ? 1u : 0u);
                    }
                    ptx::mma_commit(&empty[s]);
                }
                if (!ok) break;
                ptx::mma_commit(&zfull[zb]);
            }
            ptx::mma_commit(drain);  // completes once every MMA issued above is done
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

// ------------------------------------------------------------ GEMM1, wide bases (2K > 144)
// The same computation with the A operand in tensor memory instead of shared memory, which
// leaves shared memory to the V stages a wide basis needs (up to 2K = 256 columns).  Tensor
// memory: one Z accumulator of z_cols columns, then n_aslot A stages of 96 columns (128 frames
// x 192 K-elements, two FP16/BF16 per column).  Producer warp w owns TMEM lane quarter w % 4
// (frame rows 32 (w % 4) ..) and bin w / 4 of each 4-bin chunk and writes its cross spectra
// with tcgen05.st; the MMA reads A from tensor memory and V from a ring of n_vslot
// shared-memory stages fed by TMA.
constexpr int kAStageCols = 3 * kAtomElems / 2;   // TMEM columns of one A stage (3 atoms)
constexpr int kMaxASlots = 4, kMaxVSlots = 4;

// MMAX: bound on the microphone count (EXACT: M == MMAX, known at compile time);
// DEPTH: how many items of raw STFT values are held in registers ahead of use.
//
// Tensor memory: Z accumulators (n_zbuf buffers of z_cols columns) then n_aslot A stages of
// 96 columns (128 frames x 192 K-elements, two FP16/BF16 per column).  Producer warp w owns
// TMEM lane quarter w % 4 (frame rows 32 (w % 4) ..) and bin w / 4 of each 4-bin chunk, and
// writes its cross spectra with tcgen05.st; the MMA reads A from tensor memory and V from a
// ring of n_vslot shared-memory stages fed by TMA, so shared memory holds only V and the
// rest of the SM's 228 KB stays L1 for the STFT loads.
template <int BF16, int MMAX, bool EXACT, int DEPTH>
__global__ void __launch_bounds__(kProjThreads, 1)
    svd_proj_tm_kernel(const __grid_constant__ CUtensorMap tmap_v, const ProjParams prm) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n1 = prm.n1, n_as = prm.n_aslot, n_vs = prm.n_vslot, n_zb = prm.n_zbuf;
    const int b_stage = 3 * n1 * 128;
    const int off_bar = n_vs * b_stage;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + off_bar);
    uint64_t *full_a = bars, *empty_a = bars + kMaxASlots;
    uint64_t *full_v = bars + 2 * kMaxASlots, *empty_v = full_v + kMaxVSlots;
    uint64_t *zfull = empty_v + kMaxVSlots, *zempty = zfull + 2, *drain = zempty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(drain + 2);
    const long long budget = g_wait_budget;

    if (tid == 0) {
        for (int i = 0; i < kMaxASlots; ++i) {
            ptx::mbar_init(&full_a[i], kProdWarps);
            ptx::mbar_init(&empty_a[i], 1);
        }
        for (int i = 0; i < kMaxVSlots; ++i) {
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
    if (warp == kTmaWarp && lane == 0) ptx::prefetch_tmap(&tmap_v);
    if (warp == kMmaWarp) {
        ptx::tmem_alloc(tmem_slot, 512);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int stages_per_tile = prm.n_chunks * prm.G;
    const int my_tiles = prm.n_tiles > (int)blockIdx.x ? (prm.n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto give_up = [&]() {
        *abort_flag = 1;
        atomicOr(&g_status, 1);
    };

    if (warp < kProdWarps) {
        // -------- producers: PHAT of (frame row r, bin b) of every chunk of every tile.
        // The STFT stream of this thread is a flat sequence of items (local tile, chunk); the
        // raw values of item j + DEPTH are in flight while item j is normalised and written.
        // With EXACT, the pair layout (P, groups, slots) is known at compile time.
        constexpr int NPAIR = MMAX * (MMAX - 1) / 2;
        constexpr PairTab<MMAX> tab = make_pair_tab<MMAX>();
        const int M = EXACT ? MMAX : prm.M;
        const int P = EXACT ? NPAIR : prm.P;
        const int G = EXACT ? (NPAIR + kGroupPairs - 1) / kGroupPairs : prm.G;
        const int q4 = warp & 3, b = warp >> 2;
        const int f = q4 * 32 + lane;                      // frame row = TMEM lane
        const uint32_t lane_base = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)prm.a_col0 + (uint32_t)b;
        const int n_chunks = prm.n_chunks;
        const size_t frame_elems = (size_t)M * prm.B;
        int ld_li = 0, ld_c = 0;
        const float2 *ld_fr = prm.frames;
        bool ld_live = false;
        auto ld_seek_tile = [&]() {
            const long long frame = (long long)((int)blockIdx.x + ld_li * (int)gridDim.x) * 128 + f;
            ld_live = ld_li < my_tiles && frame < prm.T;
            ld_fr = prm.frames + (ld_live ? (size_t)frame * frame_elems : 0);
        };
        float2 raw[DEPTH][MMAX];
        auto load_next = [&](float2 (&dst)[MMAX]) {
            const int k = ld_c * kChunkBins + b;
            const bool ok = ld_live && k < prm.B;
#pragma unroll
            for (int m = 0; m < MMAX; ++m)
                dst[m] = (ok && m < M) ? ld_stream(ld_fr + (size_t)m * prm.B + k) : make_float2(0.f, 0.f);
            if (++ld_c == n_chunks) {
                ld_c = 0;
                ++ld_li;
                ld_seek_tile();
            }
        };
        ld_seek_tile();
        const int n_items = my_tiles * n_chunks;
        int st = 0;  // stage counter
        auto step = [&](float2 (&cur)[MMAX]) -> bool {
            float2 xh[MMAX];
#pragma unroll
            for (int m = 0; m < MMAX; ++m) {
                const float2 v = cur[m];
                const float mag2 = v.x * v.x + v.y * v.y;
                const float r = mag2 < 1e-30f ? 0.f : rsqrtf(mag2);
                xh[m] = make_float2(v.x * r, v.y * r);
            }
            load_next(cur);
            for (int g = 0; g < G; ++g, ++st) {
                const int s = st % n_as;
                const uint32_t par = ((st / n_as) & 1) ^ 1;
                if (ptx::warp_flag(abort_flag)) return false;
                if (!ptx::mbar_wait_warp(&empty_a[s], par, budget)) {
                    if (lane == 0) give_up();
                    return false;
                }
                ptx::tc_fence_after();
                const uint32_t col0 = lane_base + (uint32_t)(s * kAStageCols);
                const int p_lo = g * kGroupPairs;
                const int npg = min(kGroupPairs, P - p_lo);
#pragma unroll
                for (int pp = 0; pp < NPAIR; ++pp) {
                    const int i = tab.i[pp], jj = tab.j[pp];
                    if (jj < M) {
                        const int p = i * M - ((i * (i + 1)) >> 1) + (jj - i - 1);
                        const int pl = p - p_lo;
                        if (pl >= 0 && pl < npg) {
                            const float2 a0 = xh[i], b0 = xh[jj];
                            ptx::tmem_st1(col0 + (uint32_t)(pl * 4),
                                          pack2<BF16>(a0.x * b0.x + a0.y * b0.y, a0.y * b0.x - a0.x * b0.y));
                        }
                    }
                }
                if (npg & 1) ptx::tmem_st1(col0 + (uint32_t)(npg * 4), 0u);   // partner of an odd last pair
                ptx::tmem_wait_st();
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&full_a[s]);
            }
            return true;
        };
#pragma unroll
        for (int d = 0; d < DEPTH; ++d) load_next(raw[d]);
        bool ok = true;
        for (int j = 0; j < n_items && ok; j += DEPTH) {
#pragma unroll
            for (int d = 0; d < DEPTH; ++d)
                if (ok && j + d < n_items) ok = step(raw[d]);
        }
    } else if (warp < kEpiWarp0 + 4) {
        // -------- epilogue: Z of each finished tile, TMEM -> FP32 global
        const int q4 = warp - kEpiWarp0;   // TMEM lane quarter of this warp (warp % 4)
        const int r = q4 * 32 + lane;      // frame row within the tile
        for (int li = 0; li < my_tiles; ++li) {
            const int zb = n_zb == 2 ? (li & 1) : 0;
            const uint32_t zpar = n_zb == 2 ? ((li >> 1) & 1) : (li & 1);
            if (ptx::warp_flag(abort_flag)) break;
            if (!ptx::mbar_wait_warp(&zfull[zb], zpar, budget)) {
                if (lane == 0) give_up();
                break;
            }
            ptx::tc_fence_after();
            const long long frame = (long long)((int)blockIdx.x + li * (int)gridDim.x) * 128 + r;
            const bool live = frame < prm.T;
            float2 *zo = prm.z_out + (size_t)(live ? frame : 0) * prm.K;
            float zn2 = 0.f;
            for (int c0 = 0; c0 < n1; c0 += 32) {
                float v[32];
                ptx::tmem_ld32(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(zb * prm.z_cols + c0), v);
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
    } else if (warp == kTmaWarp) {
        if (lane == 0) {
            int issued = -1;
            const int n_stages = my_tiles * stages_per_tile;
            for (int st = 0; st < n_stages; ++st) {
                const int s = st % n_vs;
                if (*abort_flag) break;
                if (!ptx::mbar_wait(&empty_v[s], ((st / n_vs) & 1) ^ 1, budget)) {
                    give_up();
                    break;
                }
                const int sl = st % stages_per_tile;
                const int g = sl % prm.G;
                const int npg = min(kGroupPairs, prm.P - g * kGroupPairs);
                const int atoms = (((npg + 1) >> 1) + 3) >> 2;
                const int vcol = sl * kGroupElems;
                ptx::mbar_arrive_expect_tx(&full_v[s], (uint32_t)(atoms * n1 * 128));
                uint8_t *Bs = smem + s * b_stage;
                for (int a = 0; a < atoms; ++a)
                    for (int r0 = 0; r0 < n1; r0 += prm.v_box)   // a box spans at most 256 rows
                        ptx::tma_load_2d(Bs + a * n1 * 128 + r0 * 128, &tmap_v, &full_v[s], vcol + a * kAtomElems,
                                         r0);
                issued = st;
            }
            for (int st = max(0, issued - n_vs + 1); st <= issued; ++st)
                ptx::mbar_wait(&full_v[st % n_vs], (st / n_vs) & 1, kDrainBudget);
        }
        __syncwarp();
    } else {  // kMmaWarp
        if (lane == 0) {
            // GEMM1 N above 256 runs as two MMAs per K step: columns [0, 256) and [256, n1)
            const int nA = n1 <= 256 ? n1 : 256, nB = n1 - nA;
            const uint32_t idesc = ptx::idesc_f16(128, nA, BF16);
            const uint32_t idesc_b = ptx::idesc_f16(128, nB > 0 ? nB : 16, BF16);
            int st = 0;
            for (int li = 0; li < my_tiles; ++li) {
                const int zb = n_zb == 2 ? (li & 1) : 0;
                const uint32_t zpar = (n_zb == 2 ? ((li >> 1) & 1) : (li & 1)) ^ 1;
                if (*abort_flag) break;
                if (!ptx::mbar_wait(&zempty[zb], zpar, budget)) {
                    give_up();
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(zb * prm.z_cols);
                bool ok = true;
                for (int sl = 0; sl < stages_per_tile; ++sl, ++st) {
                    const int sa = st % n_as, sv = st % n_vs;
                    if (*abort_flag || !ptx::mbar_wait(&full_a[sa], (st / n_as) & 1, budget) ||
                        !ptx::mbar_wait(&full_v[sv], (st / n_vs) & 1, budget)) {
                        if (!*abort_flag) give_up();
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const int g = sl % prm.G;
                    const int npg = min(kGroupPairs, prm.P - g * kGroupPairs);
                    const int steps = (npg + 1) >> 1;
                    const uint32_t a_tmem = tmem + (uint32_t)(prm.a_col0 + sa * kAStageCols);
                    const uint32_t b_base = ptx::smem_u32(smem + sv * b_stage);
                    for (int k = 0; k < steps; ++k) {
                        const uint32_t bo = (k >> 2) * n1 * 128 + (k & 3) * 32;
                        ptx::mma_f16_ts(d_tmem, a_tmem + (uint32_t)(k * 8), ptx::sw128_desc(b_base + bo), idesc,
                                        (sl > 0 || k > 0) ? 1u : 0u);
                        if (nB > 0)
                            ptx::mma_f16_ts(d_tmem + (uint32_t)nA, a_tmem + (uint32_t)(k * 8),
                                            ptx::sw128_desc(b_base + bo + (uint32_t)nA * 128u), idesc_b,
                                            (sl > 0 || k > 0) ? 1u : 0u);
                    }
                    ptx::mma_commit(&empty_a[sa]);
                    ptx::mma_commit(&empty_v[sv]);
                }
                if (!ok) break;
                ptx::mma_commit(&zfull[zb]);
            }
            ptx::mma_commit(drain);  // completes once every MMA issued above is done
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

// ===================================================================== scan kernel
struct ScanParams {
    const float2 *Z;     // [T][K] complex64
    const float *zn2;    // [T] ||Z||^2
    int T, K, k2, k2_atoms, Qr, nq;
    const int32_t *rows;   // optional frame list: tile position p scans frame rows[p], p < *n_rows
    const int *n_rows;
    const int32_t *reps;
    const float2 *Dr32;  // [Qr][K] complex64, the D rows of the class representatives
    float tol_z;         // 2 * 2.1 u sqrt(L): candidate window per unit ||Z||
    float tol_abs;       // 2 * 1e-6 L
    int *ovf_count;      // frames whose window holds more than kCap classes: count, list,
    int32_t *ovf_list;   // and their argmax keys (zeroed here), for the FP32 list scan
    unsigned long long *ovf_keys;
    int32_t *idx;
    float *proj;
};

// One pass over the class tiles.  Each frame has two epilogue threads (warps w and w + 4 read
// the same TMEM lanes), one per 32-class half of every tile.  Per tile a thread takes its
// half's maximum (a tree, no branch per score), raises its running maximum m_h, and keeps every
// class of its half at or above m_h - window with its exact score in a list of kCapH; when the
// list is full the smallest of the list and the newcomer is let go and its score recorded.
// After the pass m = max(m_0, m_1) and the kept classes at or above m - window are the window
// exactly, unless a window class was let go -- which happens only when kCapH kept classes all
// score higher, i.e. when the window holds more than kCapH classes of that half; the recorded
// score tells (>= m - window), and such a frame goes to the FP32 list scan.  Neither the
// decision nor the set depends on the tile order.  Kept classes live in shared memory as
// [slot][frame] (class, score), so the 128 threads of a half touch 128 consecutive words.
// v[i] for a run-time i without local memory: a 5-level select tree on the bits of i
__device__ __forceinline__ float pick32(const float (&v)[32], int i) {
    float a[16], b[8], c[4], d[2];
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = (i & 16) ? v[k + 16] : v[k];
#pragma unroll
    for (int k = 0; k < 8; ++k) b[k] = (i & 8) ? a[k + 8] : a[k];
#pragma unroll
    for (int k = 0; k < 4; ++k) c[k] = (i & 4) ? b[k + 4] : b[k];
#pragma unroll
    for (int k = 0; k < 2; ++k) d[k] = (i & 2) ? c[k + 2] : c[k];
    return (i & 1) ? d[1] : d[0];
}

template <int BF16, int kRing>
__global__ void __launch_bounds__(kScanThreads, 2)
    svd_scan_kernel(const __grid_constant__ CUtensorMap tmap_d, const ScanParams prm) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long t0 = (long long)blockIdx.x * 128;
    const int T = prm.T;
    // tile positions [0, n_pos) are live; a CTA past them has no work (uniform exit)
    const int n_pos = prm.rows ? min(*prm.n_rows, T) : T;
    if (t0 >= n_pos) return;
    const int k2_atoms = prm.k2_atoms;
    const int b2_bytes = k2_atoms * kN2 * 128;          // one D tile
    const int off_b2 = k2_atoms * kAtomBytes;
    const int off_cand = off_b2 + kRing * b2_bytes;
    const int off_cs = off_cand + 128 * kCap * 4;
    const int off_fr = off_cs + 128 * kCap * 4;
    const int off_bar = off_fr + 128 * 4;
    int *cand = reinterpret_cast<int *>(smem + off_cand);       // [kCap][128] class (half h: slots h kCapH ..)
    float *cand_s = reinterpret_cast<float *>(smem + off_cs);   // [kCap][128] score bound
    int *fr_s = reinterpret_cast<int *>(smem + off_fr);         // frame of each row, -1 = none
    // after the pass the A operand is dead: the halves' counts and maxima go there
    int *cnt_s = reinterpret_cast<int *>(smem);                  // [2][128]
    float *mh_s = reinterpret_cast<float *>(smem + 1024);        // [2][128]
    float *dr_s = reinterpret_cast<float *>(smem + 2048);        // [2][128]
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + off_bar);
    uint64_t *b2_full = bars + 0, *b2_empty = bars + kRing, *t2_full = bars + 2 * kRing, *t2_empty = bars + 3 * kRing;
    uint64_t *drain = bars + 4 * kRing;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 4 * kRing + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 4 * kRing + 2);
    uint64_t *zbar = bars + 4 * kRing + 3;
    const long long budget = g_wait_budget;
    const int K = prm.K;

    if (tid == 0) {
        for (int i = 0; i < kRing; ++i) {
            ptx::mbar_init(&b2_full[i], 1);
            ptx::mbar_init(&b2_empty[i], 1);
            ptx::mbar_init(&t2_full[i], 1);
            ptx::mbar_init(&t2_empty[i], 32 * kScanEpiWarps);
        }
        ptx::mbar_init(drain, 1);
        ptx::mbar_init(zbar, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    if (tid < 128) {
        const long long pos = t0 + tid;
        int f = -1;
        if (pos < n_pos) {
            f = prm.rows ? prm.rows[pos] : (int)pos;
            if (!dcheck(f >= 0 && f < T, &g_status)) f = -1;
        }
        fr_s[tid] = f;
    }
    if (warp == kScanTmaWarp && lane == 0) ptx::prefetch_tmap(&tmap_d);
    if (warp == kScanMmaWarp) {
        ptx::tmem_alloc(tmem_slot, kRing * kN2);
        ptx::tmem_relinquish();
    }
    __syncthreads();
    // A operand: Z rounded to FP16/BF16, [128 frames][k2] in the 128-byte swizzle layout.  A tile
    // of consecutive frames is one contiguous run of Z: one bulk copy into the (still idle) D
    // ring, then converted from shared memory; listed frames are gathered (8 loads in flight
    // per thread).
    const int n_r = (int)min((long long)128, (long long)n_pos - t0);
    const unsigned z_bytes = (unsigned)n_r * (unsigned)K * 8u;
    const bool z_bulk = !prm.rows && (z_bytes & 15u) == 0 && z_bytes <= (unsigned)(kRing * b2_bytes);
    if (z_bulk) {
        if (tid == 0) {
            ptx::mbar_arrive_expect_tx(zbar, z_bytes);
            ptx::bulk_load(smem + off_b2, prm.Z + (size_t)t0 * K, z_bytes, zbar);
        }
        if (!ptx::mbar_wait(zbar, 0, budget)) {
            if (tid == 0) {
                *abort_flag = 1;
                atomicOr(&g_status, 1);
            }
            ptx::mbar_wait(zbar, 0, kDrainBudget);   // the copy must land before the ring is reused
        }
        const float2 *zs = reinterpret_cast<const float2 *>(smem + off_b2);
        const int per_row = k2_atoms * kAtomElems / 2;
        for (int e = tid; e < 128 * per_row; e += kScanThreads) {
            const int r = e / per_row, kk = e % per_row, n = 2 * kk;
            const float2 z = (r < n_r && kk < K) ? zs[r * K + kk] : make_float2(0.f, 0.f);
            *reinterpret_cast<uint32_t *>(smem + (n >> 6) * kAtomBytes + ptx::sw128_offset(r, n & 63)) =
                pack2<BF16>(z.x, z.y);
        }
    } else {
        const int per_row = k2_atoms * kAtomElems / 2;
        const int n_el = 128 * per_row;
        for (int e0 = tid; e0 < n_el; e0 += 8 * kScanThreads) {
            float2 z[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = e0 + u * kScanThreads;
                const int r = e / per_row, kk = e % per_row;
                const int f = e < n_el ? fr_s[r] : -1;
                z[u] = (f >= 0 && kk < K) ? prm.Z[(size_t)f * K + kk] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = e0 + u * kScanThreads;
                if (e < n_el) {
                    const int r = e / per_row, n = 2 * (e % per_row);
                    *reinterpret_cast<uint32_t *>(smem + (n >> 6) * kAtomBytes + ptx::sw128_offset(r, n & 63)) =
                        pack2<BF16>(z[u].x, z[u].y);
                }
            }
        }
    }
    ptx::fence_proxy_async_smem();
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    auto give_up = [&]() {
        *abort_flag = 1;
        atomicOr(&g_status, 1);
    };
    const int n_jobs = prm.nq;
    int my_cnt = 0;
    float my_m = 0.f, my_dropped = 0.f;

    if (warp < kScanEpiWarps) {
        const int hf = warp >> 2;               // which 32 classes of every tile
        const int r = (warp & 3) * 32 + lane;   // TMEM lane = frame row
        const int frame = fr_s[r];
        const float win = prm.tol_z * sqrtf(frame >= 0 ? prm.zn2[frame] : 0.f) + prm.tol_abs;
        const float kNaN = __int_as_float(0x7fc00000);
        float m = -__int_as_float(0x7f800000), thr = m;
        float dropped = kNaN;   // the largest score let go (NaN: none; fmaxf skips it)
        int cnt = 0;
        int *my_cand = cand + hf * kCapH * 128 + r;
        float *my_cs = cand_s + hf * kCapH * 128 + r;
        for (int j = 0; j < n_jobs; ++j) {
            const int u = j % kRing;
            const int tile = (j + (int)blockIdx.x) % prm.nq;
            if (ptx::warp_flag(abort_flag)) break;
            if (!ptx::mbar_wait_warp(&t2_full[u], (j / kRing) & 1, budget)) {
                if (lane == 0) give_up();
                break;
            }
            ptx::tc_fence_after();
            float v[32];
            ptx::tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(u * kN2 + 32 * hf), v);
            // the scores are in registers: hand the accumulator back to the MMA warp now
            ptx::tc_fence_before();
            ptx::mbar_arrive(&t2_empty[u]);
            const int qb = tile * kN2 + 32 * hf;
            const int lim = prm.Qr - qb;   // < 32 only in the last tile (NaN padding: never kept)
            if (lim < 32) {
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = i < lim ? v[i] : kNaN;
            }
            // half-tile maximum by a tree (no branch per score)
            float t[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) t[i] = fmaxf(v[i], v[i + 16]);
#pragma unroll
            for (int w = 8; w >= 1; w >>= 1) {
#pragma unroll
                for (int i = 0; i < w; ++i) t[i] = fmaxf(t[i], t[i + w]);
            }
            const float tm = t[0];
            if (tm > m) {   // new maximum: raise the window (entries now below it go at the merge)
                m = tm;
                thr = m - win;
            }
            // classes at or above the window as a bit mask (no branch per score)
            unsigned h = 0u;
#pragma unroll
            for (int i = 0; i < 32; ++i)
                if (v[i] >= thr) h |= 1u << i;
            // a lone hit is the half-tile maximum itself (tm >= it >= thr makes tm a hit too)
            const bool lone = __popc(h) == 1;
            while (h) {
                const int i = __ffs(h) - 1;
                h &= h - 1;
                float x = tm;
                if (!lone) x = pick32(v, i);
                if (cnt < kCapH) {
                    my_cand[cnt * 128] = qb + i;
                    my_cs[cnt * 128] = x;
                    ++cnt;
                } else {   // full: the smaller of x and the list's minimum (stale entries first) goes
                    int jm = 0;
                    float sm = my_cs[0];
                    for (int c = 1; c < kCapH; ++c) {
                        const float sc = my_cs[c * 128];
                        if (sc < sm) {
                            sm = sc;
                            jm = c;
                        }
                    }
                    if (x > sm) {
                        my_cand[jm * 128] = qb + i;
                        my_cs[jm * 128] = x;
                        dropped = fmaxf(dropped, sm);
                    } else {
                        dropped = fmaxf(dropped, x);
                    }
                }
            }
        }
        my_cnt = cnt;
        my_m = m;
        my_dropped = dropped;
    } else if (warp == kScanTmaWarp) {
        if (lane == 0) {
            int issued = -1;
            for (int j = 0; j < n_jobs; ++j) {
                const int u = j % kRing;
                if (*abort_flag) break;
                if (!ptx::mbar_wait(&b2_empty[u], ((j / kRing) & 1) ^ 1, budget)) {
                    give_up();
                    break;
                }
                ptx::mbar_arrive_expect_tx(&b2_full[u], (uint32_t)b2_bytes);
                uint8_t *B2 = smem + off_b2 + u * b2_bytes;
                const int tile = (j + (int)blockIdx.x) % prm.nq;  // CTAs start at different tiles
                for (int a = 0; a < k2_atoms; ++a)
                    ptx::tma_load_2d(B2 + a * kN2 * 128, &tmap_d, &b2_full[u], a * kAtomElems, tile * kN2);
                issued = j;
            }
            for (int j = max(0, issued - kRing + 1); j <= issued; ++j)
                ptx::mbar_wait(&b2_full[j % kRing], (j / kRing) & 1, kDrainBudget);
        }
        __syncwarp();
    } else if (warp == kScanMmaWarp) {
        if (lane == 0) {
            const uint32_t idesc = ptx::idesc_f16(128, kN2, BF16);
            const int steps = prm.k2 >> 4;
            const uint32_t a_base = ptx::smem_u32(smem);
            for (int j = 0; j < n_jobs; ++j) {
                const int u = j % kRing;
                const uint32_t par = (j / kRing) & 1;
                if (*abort_flag) break;
                if (!ptx::mbar_wait(&b2_full[u], par, budget) || !ptx::mbar_wait(&t2_empty[u], par ^ 1, budget)) {
                    give_up();
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t b_base = ptx::smem_u32(smem + off_b2 + u * b2_bytes);
                for (int k = 0; k < steps; ++k) {
                    const uint32_t ao = (k >> 2) * kAtomBytes + (k & 3) * 32;
                    const uint32_t bo = (k >> 2) * kN2 * 128 + (k & 3) * 32;
                    ptx::mma_f16(tmem + u * kN2, ptx::sw128_desc(a_base + ao), ptx::sw128_desc(b_base + bo), idesc,
                                 k > 0 ? 1u : 0u);
                }
                ptx::mma_commit(&b2_empty[u]);
                ptx::mma_commit(&t2_full[u]);
            }
            ptx::mma_commit(drain);
            ptx::mbar_wait(drain, 0, kDrainBudget);
        }
        __syncwarp();
    }
    __syncthreads();   // every MMA has completed: the A operand is dead
    if (warp < kScanEpiWarps) {
        const int hf = warp >> 2, r = (warp & 3) * 32 + lane;
        cnt_s[hf * 128 + r] = my_cnt;
        mh_s[hf * 128 + r] = my_m;
        dr_s[hf * 128 + r] = my_dropped;
    }
    __syncthreads();
    // merge a frame's two lists: m = max(m_0, m_1); the window is every class at or above
    // m - window.  A half that had to let a class at or above it go (list full) sends the frame
    // to the FP32 list scan; otherwise the entries at or above it are the window exactly (the
    // decision and the set do not depend on the tile order).  The merged list goes to slots
    // 0 .. n-1, its count to cnt_s[r].
    if (tid < 128 && !*abort_flag) {
        const int r = tid, frame = fr_s[r];
        const int c0 = cnt_s[r], c1 = cnt_s[128 + r];
        const float m = fmaxf(mh_s[r], mh_s[128 + r]);
        const float thr = m - (prm.tol_z * sqrtf(frame >= 0 ? prm.zn2[frame] : 0.f) + prm.tol_abs);
        int n = 0;
        if (dr_s[r] >= thr || dr_s[128 + r] >= thr) {
            n = kCap + 1;
        } else {
            for (int c = 0; c < c0 + c1; ++c) {
                const int slot = c < c0 ? c : kCapH + (c - c0);
                const float sc = cand_s[slot * 128 + r];
                if (sc >= thr) cand[(n++) * 128 + r] = cand[slot * 128 + r];
            }
        }
        cnt_s[r] = (frame >= 0 && m == m && thr == thr) ? n : 0;
    }
    __syncthreads();

    // -------- rescoring in FP32: a warp takes four frames at a time (8 lanes each); lane
    // (c, part) sums the terms k = part, part + 4, ... of candidate c, 2 candidates per round
    // (frames carry 1-2 candidates on typical inputs).  The terms of a 64-term block are
    // loaded in one unrolled batch from the class-indexed D copy, so a round costs one L2
    // round trip; the class becomes a direction index once, at the end.
    if (!*abort_flag) {
        const int g4 = lane >> 3, c2 = (lane >> 2) & 1, part = lane & 3;
        for (int r0 = 4 * warp; r0 < 128; r0 += 4 * (kScanThreads / 32)) {
            const int r = r0 + g4;
            const int frame = fr_s[r];
            const bool live = frame >= 0;
            const int n = live ? cnt_s[r] : 0;
            const int total = n <= kCap ? n : 0;   // n > kCap: the FP32 list scan takes the frame
            const float2 *zr = prm.Z + (size_t)(live ? frame : 0) * K;
            float best = 0.f;
            int bc = -1;
            int tmax = max(total, __shfl_xor_sync(0xffffffffu, total, 8));
            tmax = max(tmax, __shfl_xor_sync(0xffffffffu, tmax, 16));
            for (int base = 0; base < tmax; base += 2) {
                const int c = base + c2;
                int cls = -1;
                if (c < total) {
                    const int v = cand[c * 128 + r];
                    if (dcheck(v >= 0 && v < prm.Qr, &g_status)) cls = v;
                }
                float acc = 0.f;
                if (cls >= 0) {
                    const float2 *dq = prm.Dr32 + (size_t)cls * K;
                    for (int k0 = 0; k0 < K; k0 += 64) {
                        float2 d[16], z[16];
#pragma unroll
                        for (int u = 0; u < 16; ++u) {
                            const int kk = k0 + part + 4 * u;
                            d[u] = kk < K ? __ldg(dq + kk) : make_float2(0.f, 0.f);
                            z[u] = kk < K ? __ldg(zr + kk) : make_float2(0.f, 0.f);
                        }
#pragma unroll
                        for (int u = 0; u < 16; ++u) {
                            if (k0 + part + 4 * u < K) {
                                acc = fmaf(d[u].x, z[u].x, acc);
                                acc = fmaf(-d[u].y, z[u].y, acc);
                            }
                        }
                    }
                }
                acc += __shfl_xor_sync(0xffffffffu, acc, 1);
                acc += __shfl_xor_sync(0xffffffffu, acc, 2);
                // classes are numbered in increasing order of their representative direction,
                // so the lowest class of a tie is the lowest direction index
                if (cls >= 0 && (bc < 0 || acc > best || (acc == best && cls < bc))) {
                    best = acc;
                    bc = cls;
                }
            }
            // best over the 2 candidate groups of this 8-lane group
            {
                const float ov = __shfl_xor_sync(0xffffffffu, best, 4);
                const int oc = __shfl_xor_sync(0xffffffffu, bc, 4);
                const bool take = (bc < 0) || (oc >= 0 && (ov > best || (ov == best && oc < bc)));
                if (take) {
                    best = ov;
                    bc = oc;
                }
            }
            if ((lane & 7) == 0 && live) {
                if (n > kCap) {
                    const int pos = atomicAdd(prm.ovf_count, 1);
                    prm.ovf_list[pos] = (int32_t)frame;
                    prm.ovf_keys[pos] = 0ull;
                } else {
                    prm.idx[frame] = bc < 0 ? -1 : __ldg(prm.reps + bc);
                    if (prm.proj) prm.proj[frame] = bc < 0 ? __int_as_float(0x7fc00000) : best;
                }
            }
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == kScanMmaWarp) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, kRing * kN2);
    }
}

// =================================================================== host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

int encode_tmap_2d(CUtensorMap *map, void *base, int bf16, uint64_t inner, uint64_t rows,
                   uint32_t box_inner, uint32_t box_rows) {
    EncodeTiledFn enc = get_encode();
    SP_CHECK(enc != nullptr, SP_ECUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {inner * 2};
    cuuint32_t box[2] = {box_inner, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, base,
                     dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    SP_CHECK(r == CUDA_SUCCESS, SP_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return SP_OK;
}

int encode_tmap_f32_2d(CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows, uint64_t row_stride_bytes,
                       uint32_t box_inner, uint32_t box_rows) {
    EncodeTiledFn enc = get_encode();
    SP_CHECK(enc != nullptr, SP_ECUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {row_stride_bytes};
    cuuint32_t box[2] = {box_inner, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    SP_CHECK(r == CUDA_SUCCESS, SP_ECUDA, "cuTensorMapEncodeTiled (f32) failed (" + std::to_string((int)r) + ")");
    return SP_OK;
}

struct TcMaps {
    CUtensorMap v[2], d[2], vbm[2];
    bool has_vbm = false;
};

int tc_prepare(sp_basis *b) {
    const sp_steering *st = b->st;
    const int K = b->K, P = st->P, B = st->B, L = st->L;
    TcLayout t = make_tc_layout(P, B, K);
    t.v_box = t.n1 <= 256 ? t.n1 : t.n1 / 2;   // a TMA box spans at most 256 rows
    b->tc = t;
    if (t.n1 > kMaxN1 || st->M > 16) {
        b->tc.n1 = 0;  // tensor-core path unavailable for this basis
        return SP_OK;
    }
    const int G = (P + kGroupPairs - 1) / kGroupPairs;
    b->v_scale = (float)std::sqrt((double)L);
    const size_t nv = (size_t)t.n1 * t.row_elems;
    std::vector<float> vf(nv, 0.f);
    for (int c = 0; c < t.n_chunks; ++c)
        for (int g = 0; g < G; ++g)
            for (int pl = 0; pl < kGroupPairs; ++pl) {
                const int p = g * kGroupPairs + pl;
                if (p >= P) break;
                for (int bb = 0; bb < kChunkBins; ++bb) {
                    const int k = c * kChunkBins + bb;
                    if (k >= B) break;
                    const size_t l = (size_t)p * B + k;
                    const size_t e = (size_t)(c * G + g) * kGroupElems + pl * 8 + 2 * bb;
                    for (int kk = 0; kk < K; ++kk) {
                        const double vr = b->V[(l * K + kk) * 2] * b->v_scale;
                        const double vi = b->V[(l * K + kk) * 2 + 1] * b->v_scale;
                        vf[(size_t)(2 * kk) * t.row_elems + e] = (float)vr;
                        vf[(size_t)(2 * kk) * t.row_elems + e + 1] = (float)vi;
                        vf[(size_t)(2 * kk + 1) * t.row_elems + e] = (float)-vi;
                        vf[(size_t)(2 * kk + 1) * t.row_elems + e + 1] = (float)vr;
                    }
                }
            }
    // bin-major copy for the TMA-fed GEMM1 of 7-microphone arrays (P = 21 <= 24: one stage per
    // chunk; pair p, bin bb of chunk c at element c * 192 + 48 bb + 2 p)
    const bool bm = st->M == 7 && (B & 1) && t.n1 <= 224;
    std::vector<float> vbm;
    if (bm) {
        vbm.assign(nv, 0.f);
        for (int c = 0; c < t.n_chunks; ++c)
            for (int p = 0; p < P; ++p)
                for (int bb = 0; bb < kChunkBins; ++bb) {
                    const int k = c * kChunkBins + bb;
                    if (k >= B) break;
                    const size_t l = (size_t)p * B + k;
                    const size_t e = (size_t)c * kGroupElems + 48 * bb + 2 * p;
                    for (int kk = 0; kk < K; ++kk) {
                        const double vr = b->V[(l * K + kk) * 2] * b->v_scale;
                        const double vi = b->V[(l * K + kk) * 2 + 1] * b->v_scale;
                        vbm[(size_t)(2 * kk) * t.row_elems + e] = (float)vr;
                        vbm[(size_t)(2 * kk) * t.row_elems + e + 1] = (float)vi;
                        vbm[(size_t)(2 * kk + 1) * t.row_elems + e] = (float)-vi;
                        vbm[(size_t)(2 * kk + 1) * t.row_elems + e + 1] = (float)vr;
                    }
                }
    }
    const int dcols = t.k2_atoms * kAtomElems;
    const int Qr = (int)st->reps.size();
    std::vector<float> df((size_t)Qr * dcols, 0.f);
    for (int r = 0; r < Qr; ++r) {
        const size_t q = (size_t)st->reps[r];
        for (int kk = 0; kk < K; ++kk) {
            df[(size_t)r * dcols + 2 * kk] = (float)b->D[(q * K + kk) * 2];
            df[(size_t)r * dcols + 2 * kk + 1] = (float)-b->D[(q * K + kk) * 2 + 1];
        }
    }
    TcMaps *maps = new TcMaps();
    for (int prec = 0; prec < 2; ++prec) {
        std::vector<uint16_t> hv(nv), hd(df.size());
        for (size_t i = 0; i < nv; ++i) {
            if (prec == 0) { __half h = __float2half_rn(vf[i]); hv[i] = *reinterpret_cast<uint16_t *>(&h); }
            else { __nv_bfloat16 h = __float2bfloat16_rn(vf[i]); hv[i] = *reinterpret_cast<uint16_t *>(&h); }
        }
        for (size_t i = 0; i < df.size(); ++i) {
            if (prec == 0) { __half h = __float2half_rn(df[i]); hd[i] = *reinterpret_cast<uint16_t *>(&h); }
            else { __nv_bfloat16 h = __float2bfloat16_rn(df[i]); hd[i] = *reinterpret_cast<uint16_t *>(&h); }
        }
        SP_TRY(b->Vtc[prec].reserve(nv * 2));
        SP_TRY(b->Dtc[prec].reserve(hd.size() * 2));
        SP_CUDA(cudaMemcpy(b->Vtc[prec].p, hv.data(), nv * 2, cudaMemcpyHostToDevice));
        SP_CUDA(cudaMemcpy(b->Dtc[prec].p, hd.data(), hd.size() * 2, cudaMemcpyHostToDevice));
        int rc = encode_tmap_2d(&maps->v[prec], b->Vtc[prec].p, prec, t.row_elems, t.n1, kAtomElems, t.v_box);
        if (rc == SP_OK) rc = encode_tmap_2d(&maps->d[prec], b->Dtc[prec].p, prec, dcols, Qr, kAtomElems, kN2);
        if (rc == SP_OK && bm) {
            for (size_t i = 0; i < nv; ++i) {
                if (prec == 0) { __half h = __float2half_rn(vbm[i]); hv[i] = *reinterpret_cast<uint16_t *>(&h); }
                else { __nv_bfloat16 h = __float2bfloat16_rn(vbm[i]); hv[i] = *reinterpret_cast<uint16_t *>(&h); }
            }
            rc = b->Vbm[prec].reserve(nv * 2);
            if (rc == SP_OK && cudaMemcpy(b->Vbm[prec].p, hv.data(), nv * 2, cudaMemcpyHostToDevice) != cudaSuccess)
                rc = fail(SP_ECUDA, "tc_prepare: copy of the bin-major V");
            if (rc == SP_OK)
                rc = encode_tmap_2d(&maps->vbm[prec], b->Vbm[prec].p, prec, t.row_elems, t.n1, kAtomElems, t.v_box);
            maps->has_vbm = rc == SP_OK;
        }
        if (rc != SP_OK) {
            delete maps;
            return rc;
        }
    }
    b->tc_maps = maps;
    return SP_OK;
}

const CUtensorMap *tc_vmap_binmajor(const sp_basis *b, int bf16) {
    const TcMaps *m = reinterpret_cast<const TcMaps *>(b->tc_maps);
    return m && m->has_vbm ? &m->vbm[bf16 ? 1 : 0] : nullptr;
}

void tc_release(sp_basis *b) {
    delete reinterpret_cast<TcMaps *>(b->tc_maps);
    b->tc_maps = nullptr;
}

using ProjKernel = void (*)(CUtensorMap, ProjParams);
using ScanKernel = void (*)(CUtensorMap, ScanParams);

// The GEMM1 variant for a basis: A operand in shared memory (2K <= 144) or in tensor memory,
// exactly 7 microphones (the Table 2 arrays), up to 8, up to 16.
static ProjKernel proj_kernel_for(const TcLayout &t, int bf, int M) {
    static const ProjKernel smem_k[6] = {
        svd_proj_kernel<0, 7, true, 2>, svd_proj_kernel<0, 8, false, 2>, svd_proj_kernel<0, 16, false, 1>,
        svd_proj_kernel<1, 7, true, 2>, svd_proj_kernel<1, 8, false, 2>, svd_proj_kernel<1, 16, false, 1>};
    static const ProjKernel tm_k[6] = {
        svd_proj_tm_kernel<0, 7, true, 2>, svd_proj_tm_kernel<0, 8, false, 2>, svd_proj_tm_kernel<0, 16, false, 1>,
        svd_proj_tm_kernel<1, 7, true, 2>, svd_proj_tm_kernel<1, 8, false, 2>, svd_proj_tm_kernel<1, 16, false, 1>};
    const int which = bf * 3 + (M == 7 ? 0 : M <= 8 ? 1 : 2);
    return t.n1 <= kMaxN1Smem ? smem_k[which] : tm_k[which];
}

// D tiles in flight of the scan: four, two when the Z tile and four D tiles would not fit (2K > 256)
static int scan_smem_bytes(const TcLayout &t, int ring) {
    return t.k2_atoms * kAtomBytes + ring * t.k2_atoms * kN2 * 128 + 2 * 128 * kCap * 4 + 128 * 4 +
           (4 * ring + 4) * 8 + 1024;
}
static int scan_ring_for(const TcLayout &t) {
    return scan_smem_bytes(t, kRingMax) <= 232448 ? kRingMax : 2;
}

static ScanKernel scan_kernel_for(const TcLayout &t, int bf) {
    static const ScanKernel k[4] = {svd_scan_kernel<0, kRingMax>, svd_scan_kernel<0, 2>, svd_scan_kernel<1, kRingMax>,
                                    svd_scan_kernel<1, 2>};
    return k[bf * 2 + (scan_ring_for(t) == kRingMax ? 0 : 1)];
}

int prepare_tc(const sp_basis *b, int prec) {
    const TcLayout &t = b->tc;
    if (t.n1 <= 0 || !b->tc_maps) return SP_OK;
    const int bf = prec == SP_PREC_BF16 ? 1 : 0;
    cudaFuncAttributes a;
    const void *k1 = (const void *)proj_kernel_for(t, bf, b->st->M);
    const void *k2 = (const void *)scan_kernel_for(t, bf);
    SP_CUDA(cudaFuncGetAttributes(&a, k1));
    SP_CUDA(cudaFuncGetAttributes(&a, k2));
    SP_TRY(ensure_max_smem(k1));
    return ensure_max_smem(k2);
}

int launch_svd_proj(const sp_basis *b, const void *frames, int T, int prec, void *z_out, float *zn2_out,
                    cudaStream_t s, int max_ctas, int proj_variant) {
    if (T == 0) return SP_OK;
    const TcLayout &t = b->tc;
    SP_CHECK(t.n1 > 0 && b->tc_maps, SP_ENOTIMPL,
             "tensor-core path supports 2K <= 288 and M <= 16 (use SP_PREC_FP32)");
    const int bf = prec == SP_PREC_BF16 ? 1 : 0;
    const TcMaps *maps = reinterpret_cast<const TcMaps *>(b->tc_maps);
    ProjParams p;
    p.frames = (const float2 *)frames;
    p.T = T;
    p.M = b->st->M;
    p.B = b->st->B;
    p.P = b->st->P;
    p.G = (p.P + kGroupPairs - 1) / kGroupPairs;
    p.n_chunks = t.n_chunks;
    p.n1 = t.n1;
    p.K = b->K;
    p.inv_vscale = 1.f / b->v_scale;
    p.z_out = (float2 *)z_out;
    p.zn2_out = zn2_out;
    p.n_tiles = (int)(((long long)T + 127) / 128);
    const int grid = std::min(p.n_tiles, max_ctas > 0 ? std::min(max_ctas, num_sms()) : num_sms());
    if (proj_variant == 0) {   // the TMA-fed kernel for 7-microphone arrays where its plan applies
        const int rc = launch_svd_proj_tma(b, frames, T, prec, z_out, zn2_out, s, max_ctas);
        if (rc != SP_ENOTIMPL) return rc;
    }
    const ProjKernel kern = proj_kernel_for(t, bf, p.M);
    if (t.n1 <= kMaxN1Smem) {
        // A operand in shared memory: two stages of A (48 KB) and V (3 atoms of n1 rows)
        const int smem = 2 * 3 * kAtomBytes + 2 * 3 * t.n1 * 128 + 128 + 1024;
        SP_CHECK(smem <= 232448, SP_ENOTIMPL, "shared-memory plan exceeds 227 KB");
        SP_TRY(ensure_max_smem((const void *)kern));
        // at least 120 KB so that one CTA (holding all 512 TMEM columns) runs per SM
        const int smem_launch = std::max(smem, 120 * 1024);
        kern<<<grid, kProjThreads, smem_launch, s>>>(maps->v[bf], p);
    } else {
        // A operand in tensor memory: one Z buffer, then A stages; shared memory holds V only
        p.z_cols = (t.n1 + 31) / 32 * 32;
        p.n_zbuf = 1;
        p.a_col0 = p.z_cols;
        p.n_aslot = std::min(kMaxASlots, (512 - p.a_col0) / kAStageCols);
        const int b_stage = 3 * t.n1 * 128;
        p.n_vslot = std::min(kMaxVSlots, (216 * 1024) / b_stage);
        p.v_box = t.v_box;
        SP_CHECK(p.n_aslot >= 2 && p.n_vslot >= 2, SP_ENOTIMPL, "tensor-core plan: too few pipeline stages");
        const int smem = p.n_vslot * b_stage + 256 + 1024;
        SP_CHECK(smem <= 232448, SP_ENOTIMPL, "shared-memory plan exceeds 227 KB");
        SP_TRY(ensure_max_smem((const void *)kern));
        kern<<<grid, kProjThreads, std::max(smem, 120 * 1024), s>>>(maps->v[bf], p);
    }
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

size_t scan_workspace_bytes(int T) { return 256 + ((size_t)T * 4 + 255) / 256 * 256 + (size_t)T * 8; }

int launch_svd_scan(const sp_basis *b, const void *Z, const float *zn2, int T, int prec, int32_t *idx,
                    float *proj, cudaStream_t s, void *ws, const int32_t *rows, const int *n_rows) {
    if (T == 0) return SP_OK;
    SP_CHECK(ws && (reinterpret_cast<uintptr_t>(ws) & 255) == 0, SP_EINVAL, "scan: workspace missing or misaligned");
    const TcLayout &t = b->tc;
    SP_CHECK(t.n1 > 0 && b->tc_maps, SP_ENOTIMPL,
             "tensor-core path supports 2K <= 288 and M <= 16 (use SP_PREC_FP32)");
    const int bf = prec == SP_PREC_BF16 ? 1 : 0;
    const TcMaps *maps = reinterpret_cast<const TcMaps *>(b->tc_maps);
    ScanParams p;
    p.Z = (const float2 *)Z;
    p.zn2 = zn2;
    p.T = T;
    p.K = b->K;
    p.k2 = t.k2;
    p.k2_atoms = t.k2_atoms;
    p.Qr = (int)b->st->reps.size();
    p.nq = (p.Qr + kN2 - 1) / kN2;
    p.reps = b->st->d_reps.as<int32_t>();
    p.Dr32 = b->Dc32r.as<float2>();
    p.rows = rows;
    p.n_rows = n_rows;
    const double u = bf ? std::ldexp(1.0, -8) : std::ldexp(1.0, -11);  // unit roundoff
    const double L = (double)b->st->L;
    p.tol_z = (float)(2.0 * 2.1 * u * std::sqrt(L));
    p.tol_abs = (float)(2.0 * 1e-6 * L);
    p.idx = idx;
    p.proj = proj;
    char *w = static_cast<char *>(ws);
    p.ovf_count = reinterpret_cast<int *>(w);
    p.ovf_list = reinterpret_cast<int32_t *>(w + 256);
    p.ovf_keys = reinterpret_cast<unsigned long long *>(w + 256 + ((size_t)T * 4 + 255) / 256 * 256);
    SP_CUDA(cudaMemsetAsync(p.ovf_count, 0, sizeof(int), s));
    const int ring = scan_ring_for(t);
    const int smem = scan_smem_bytes(t, ring);
    SP_CHECK(smem <= 232448, SP_ENOTIMPL, "scan: shared-memory plan exceeds 227 KB");
    const ScanKernel kern = scan_kernel_for(t, bf);
    SP_TRY(ensure_max_smem((const void *)kern));
    const unsigned grid = (unsigned)(((long long)T + 127) / 128);
    kern<<<grid, kScanThreads, smem, s>>>(maps->d[bf], p);
    SP_CUDA(cudaGetLastError());
    // frames with more than kCap classes in their window: the exact FP32 scan over every class
    return launch_svd_scan_f32_list(b, Z, T, p.ovf_count, p.ovf_list, reinterpret_cast<uint64_t *>(p.ovf_keys), idx,
                                    proj, s);
}

}  // namespace sp

extern "C" int sp_set_wait_budget(long long cycles) {
    using namespace sp;
    const long long v = cycles <= 0 ? 2000000000LL : cycles;
    SP_CUDA(cudaMemcpyToSymbol(g_wait_budget, &v, sizeof(v)));
    h_wait_budget = v;
    return SP_OK;
}
