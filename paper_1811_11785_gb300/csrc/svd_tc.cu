// Tensor-core SVD-PHAT (online steps 1-3 of Algorithm 1) in one kernel, sm_103a.
//
//   GEMM1 (Eq. 12):  Z^T = X^T conj(V) as a real GEMM over 2L, M = 128 frames per CTA,
//                    N = 2K (Re Z_k, Im Z_k interleaved), FP16 or BF16 inputs, FP32
//                    accumulator in TMEM.  The A operand (the PHAT cross spectra, Eq. 3)
//                    is produced straight into shared memory by 8 producer warps from the
//                    STFT frames; X never reaches global memory.  The B operand (V, scaled
//                    by sqrt(L)) streams from L2 by TMA.
//   GEMM2 (Eq. 14):  Y = Re{D Z} = [Re D, -Im D] . [Re Z, Im Z] over Q tiles of 128,
//                    FP16/BF16 inputs (Z rounded from the FP32 accumulator), FP32 in
//                    TMEM.  Y never leaves the chip: each frame's thread keeps the 8 best
//                    (score, q) pairs.
//   Rescoring:       the 8 candidates are rescored in FP32 from FP32 Z and FP32 D; the best
//                    one (ties -> lowest q) is the frame's direction.
//
// K-dimension layout of GEMM1 (a permutation of the paper's column order p*B + k): the
// contraction is cut into stages (bin chunk c of 4 bins, pair group g of <= 24 pairs);
// in a stage, pair p (local index) and bin b sit at elements p*8 + 2b (real) and
// p*8 + 2b + 1 (imaginary), so one K16 MMA step covers 2 pairs x 4 bins and a 64-element
// 128-byte-swizzled atom covers 8 pairs.
//
// Warp roles (384 threads): warps 0-7 produce A tiles (and warps 0-3 are the epilogue),
// warp 8 issues TMA loads, warp 9 allocates TMEM and issues the MMAs.  Every mbarrier
// wait is bounded; a wait that gives up records an error in g_status and the CTA drains
// its in-flight copies/MMAs (with a fixed generous bound) and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.h"
#include "ptx.cuh"

namespace sp {

__device__ int g_status = 0;
__device__ long long g_wait_budget = 2000000000LL;  // SM cycles per bounded wait
constexpr long long kDrainBudget = 4000000000LL;     // draining in-flight async work

static long long h_wait_budget = 2000000000LL;
long long wait_budget() { return h_wait_budget; }

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
constexpr int kMaxN1 = 144;           // GEMM1 N limit of this shared-memory plan
constexpr int kThreads = 384;
constexpr int kProducerThreads = 256;
constexpr int kTmemCols = 512;
constexpr int kTmemY = 256;           // GEMM2 accumulators at columns 256 and 384
constexpr int kTop = 8;

TcLayout make_tc_layout(int P, int B, int K) {
    TcLayout t;
    t.P = P;
    t.Pp = (P + 1) / 2 * 2;
    t.steps_per_chunk = 0;   // per group, computed in the kernel
    t.atoms_per_chunk = 3;
    t.n_chunks = (B + kChunkBins - 1) / kChunkBins;
    const int G = (P + kGroupPairs - 1) / kGroupPairs;
    t.row_elems = t.n_chunks * G * kGroupElems;
    t.n1 = (2 * K + 15) / 16 * 16;
    t.k2 = (2 * K + 15) / 16 * 16;
    t.k2_atoms = (t.k2 + kAtomElems - 1) / kAtomElems;
    t.n2 = 128;
    return t;
}

struct TcParams {
    const float2 *frames;
    int T, M, B, P, G, n_chunks;
    int n1, K, Q, k2, k2_atoms, nq;
    float inv_vscale;
    int do_scan;
    const float2 *Dc32;  // [Q][K] complex64
    int32_t *idx;
    float *proj;
    float2 *z_out;       // [T][K] complex64 or null
};

struct SmemPlan {
    int a_stage, b_stage;          // bytes per GEMM1 stage buffer
    int off_b;                     // offset of the B stages
    int off_a2, off_b2, off_zf;    // GEMM2 regions (overlap GEMM1)
    int zstride;                   // floats per Zf row
    int off_bar;                   // barriers
    int total;
};

static SmemPlan make_plan(const TcLayout &t) {
    SmemPlan p;
    p.a_stage = 3 * kAtomBytes;
    p.b_stage = 3 * t.n1 * 128;
    p.off_b = 2 * p.a_stage;
    const int r0 = p.off_b + 2 * p.b_stage;
    p.off_a2 = 0;
    p.off_b2 = t.k2_atoms * kAtomBytes;
    p.off_zf = p.off_b2 + 2 * t.k2_atoms * kAtomBytes;
    p.zstride = t.n1 + 1;
    const int r1 = p.off_zf + 128 * p.zstride * 4;
    p.off_bar = (std::max(r0, r1) + 127) / 128 * 128;
    p.total = p.off_bar + 256 + 1024;  // + slack for 1024-byte alignment
    // at least 120 KB so that one CTA (holding all 512 TMEM columns) runs per SM
    p.total = std::max(p.total, 120 * 1024);
    return p;
}

__device__ __forceinline__ float2 ld_stream(const float2 *p) {
    float2 v;
    asm volatile("ld.global.nc.L2::256B.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}


// The 120 pairs (i, j), i < j < 16, in Eq. 7 order; unrolled loops over this table keep
// every x^_m access a compile-time register index.
struct PairTab { int i[120]; int j[120]; };
constexpr PairTab make_pair_tab() {
    PairTab t{};
    int n = 0;
    for (int i = 0; i < 16; ++i)
        for (int j = i + 1; j < 16; ++j) { t.i[n] = i; t.j[n] = j; ++n; }
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

template <int BF16>
__global__ void __launch_bounds__(kThreads, 1)
    svd_tc_kernel(const __grid_constant__ CUtensorMap tmap_v, const __grid_constant__ CUtensorMap tmap_d,
                  const TcParams prm) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // shared-memory plan (mirrors make_plan on the host)
    const int n1 = prm.n1;
    const int a_stage = 3 * kAtomBytes, b_stage = 3 * n1 * 128;
    const int off_b = 2 * a_stage;
    const int off_b2 = prm.k2_atoms * kAtomBytes;
    const int off_zf = off_b2 + 2 * prm.k2_atoms * kAtomBytes;
    const int zstride = n1 + 1;
    const int r0 = off_b + 2 * b_stage, r1 = off_zf + 128 * zstride * 4;
    const int off_bar = (max(r0, r1) + 127) / 128 * 128;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + off_bar);
    uint64_t *full_a = bars + 0, *full_b = bars + 2, *empty = bars + 4, *g1_done = bars + 6;
    uint64_t *b2_full = bars + 7, *b2_empty = bars + 9, *t2_full = bars + 11, *t2_empty = bars + 13;
    uint64_t *drain = bars + 15;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 16);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 17);

    const long long budget = g_wait_budget;
    const long long t0 = (long long)blockIdx.x * 128;

    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(&full_a[i], kProducerThreads);
            ptx::mbar_init(&full_b[i], 1);
            ptx::mbar_init(&empty[i], 1);
            ptx::mbar_init(&b2_full[i], 1);
            ptx::mbar_init(&b2_empty[i], 1);
            ptx::mbar_init(&t2_full[i], 1);
            ptx::mbar_init(&t2_empty[i], 128);
        }
        ptx::mbar_init(g1_done, 1);
        ptx::mbar_init(drain, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    if (warp == 8 && lane == 0) {
        ptx::prefetch_tmap(&tmap_v);
        ptx::prefetch_tmap(&tmap_d);
    }
    if (warp == 9) {
        ptx::tmem_alloc(tmem_slot, kTmemCols);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int n_stages = prm.n_chunks * prm.G;
    bool drained = false;  // MMA issuer: all issued MMAs known complete

    auto give_up = [&]() {
        *abort_flag = 1;
        atomicOr(&g_status, 1);
    };

    // =============================================================== GEMM1
    if (warp < 8) {
        // ---------------- producers: PHAT of (frame f, bins 2bp, 2bp+1) of each chunk
        const int f = tid >> 1, bp = tid & 1;
        const long long frame = t0 + f;
        const bool live = frame < prm.T;
        const float2 *fr = prm.frames + (size_t)(live ? frame : 0) * prm.M * prm.B;
        for (int c = 0; c < prm.n_chunks; ++c) {
            float2 xh[16][2];
#pragma unroll
            for (int m = 0; m < 16; ++m) {
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    xh[m][b] = make_float2(0.f, 0.f);
                    const int k = c * kChunkBins + 2 * bp + b;
                    if (m < prm.M && live && k < prm.B) {
                        const float2 v = ld_stream(fr + (size_t)m * prm.B + k);
                        const float mag2 = v.x * v.x + v.y * v.y;
                        const float r = mag2 < 1e-30f ? 0.f : rsqrtf(mag2);
                        xh[m][b] = make_float2(v.x * r, v.y * r);
                    }
                }
            }
            for (int g = 0; g < prm.G; ++g) {
                const int st = c * prm.G + g;
                const int s = st & 1;
                const uint32_t par = ((st >> 1) & 1) ^ 1;
                if (*abort_flag) break;
                if (!ptx::mbar_wait(&empty[s], par, budget)) {
                    give_up();
                    break;
                }
                uint8_t *A = smem + s * a_stage;
                const int p_lo = g * kGroupPairs;
                const int npg = min(kGroupPairs, prm.P - p_lo);
                const int nslots = (npg + 1) & ~1;  // even number of pair slots written
#pragma unroll
                for (int pp = 0; pp < 120; ++pp) {
                    constexpr PairTab tab = make_pair_tab(); const int i = tab.i[pp], j = tab.j[pp];
                    if (j < prm.M) {
                        const int p = i * prm.M - ((i * (i + 1)) >> 1) + (j - i - 1);
                        const int pl = p - p_lo;
                        if (pl >= 0 && pl < npg) {
                            const float2 a0 = xh[i][0], b0 = xh[j][0];
                            const float2 a1 = xh[i][1], b1 = xh[j][1];
                            const uint32_t w0 = pack2<BF16>(a0.x * b0.x + a0.y * b0.y, a0.y * b0.x - a0.x * b0.y);
                            const uint32_t w1 = pack2<BF16>(a1.x * b1.x + a1.y * b1.y, a1.y * b1.x - a1.x * b1.y);
                            const uint32_t off = (pl >> 3) * kAtomBytes + f * 128 +
                                                 (((pl & 7) ^ (f & 7)) << 4) + bp * 8;
                            asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(ptx::smem_u32(A + off)),
                                         "r"(w0), "r"(w1)
                                         : "memory");
                        }
                    }
                }
                if (nslots > npg) {  // zero partner of an odd last pair
                    const int pl = npg;
                    const uint32_t off = (pl >> 3) * kAtomBytes + f * 128 + (((pl & 7) ^ (f & 7)) << 4) + bp * 8;
                    asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(ptx::smem_u32(A + off)), "r"(0u), "r"(0u)
                                 : "memory");
                }
                ptx::fence_proxy_async_smem();
                ptx::mbar_arrive(&full_a[s]);
            }
            if (*abort_flag) break;
        }
    } else if (warp == 8) {
        // ---------------- TMA producer for V tiles
        if (lane == 0) {
            int issued_stage = -1;
            for (int st = 0; st < n_stages; ++st) {
                const int s = st & 1;
                const uint32_t par = ((st >> 1) & 1) ^ 1;
                if (*abort_flag) break;
                if (!ptx::mbar_wait(&empty[s], par, budget)) {
                    give_up();
                    break;
                }
                const int g = st % prm.G;
                const int npg = min(kGroupPairs, prm.P - g * kGroupPairs);
                const int steps = (npg + 1) >> 1;
                const int atoms = (steps + 3) >> 2;
                ptx::mbar_arrive_expect_tx(&full_b[s], (uint32_t)(atoms * n1 * 128));
                uint8_t *Bs = smem + off_b + s * b_stage;
                for (int a = 0; a < atoms; ++a)
                    ptx::tma_load_2d(Bs + a * n1 * 128, &tmap_v, &full_b[s], st * kGroupElems + a * kAtomElems, 0);
                issued_stage = st;
            }
            // drain: wait for the last issued loads of both buffers to land
            for (int st = max(0, issued_stage - 1); st <= issued_stage; ++st)
                ptx::mbar_wait(&full_b[st & 1], (st >> 1) & 1, kDrainBudget);
        }
        __syncwarp();
    } else if (warp == 9) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = ptx::idesc_f16(128, n1, BF16);
            bool ok = true;
            for (int st = 0; st < n_stages && ok; ++st) {
                const int s = st & 1;
                const uint32_t par = (st >> 1) & 1;
                if (*abort_flag) { ok = false; break; }
                if (!ptx::mbar_wait(&full_a[s], par, budget) || !ptx::mbar_wait(&full_b[s], par, budget)) {
                    give_up();
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const int g = st % prm.G;
                const int npg = min(kGroupPairs, prm.P - g * kGroupPairs);
                const int steps = (npg + 1) >> 1;
                const uint32_t a_base = ptx::smem_u32(smem + s * a_stage);
                const uint32_t b_base = ptx::smem_u32(smem + off_b + s * b_stage);
                for (int k = 0; k < steps; ++k) {
                    const uint32_t ao = (k >> 2) * kAtomBytes + (k & 3) * 32;
                    const uint32_t bo = (k >> 2) * n1 * 128 + (k & 3) * 32;
                    ptx::mma_f16(tmem, ptx::sw128_desc(a_base + ao), ptx::sw128_desc(b_base + bo), idesc,
                                 (st > 0 || k > 0) ? 1u : 0u);
                }
                ptx::mma_commit(&empty[s]);
            }
            if (ok) {
                ptx::mma_commit(g1_done);
            } else {
                ptx::mma_commit(drain);
                ptx::mbar_wait(drain, 0, kDrainBudget);
                drained = true;
            }
        }
        __syncwarp();
    }

    // =============================================================== epilogue 1: Z
    float *Zf = reinterpret_cast<float *>(smem + off_zf);
    if (warp < 4) {
        const int r = tid;  // TMEM lane = frame row
        bool ok = !*abort_flag && ptx::mbar_wait(g1_done, 0, budget);
        if (!ok && !*abort_flag) give_up();
        if (ok) {
            ptx::tc_fence_after();
            const long long frame = t0 + r;
            uint8_t *A2 = smem;  // GEMM2 A operand, k2_atoms atoms
            for (int c0 = 0; c0 < n1; c0 += 32) {
                float v[32];
                ptx::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
                for (int i = 0; i < 32; i += 2) {
                    const int n = c0 + i;
                    const float zr = v[i] * prm.inv_vscale, zi = v[i + 1] * prm.inv_vscale;
                    const bool in = n < 2 * prm.K;
                    Zf[r * zstride + n] = in ? zr : 0.f;
                    Zf[r * zstride + n + 1] = in ? zi : 0.f;
                    const uint32_t w = pack2<BF16>(in ? zr : 0.f, in ? zi : 0.f);
                    const uint32_t off = (n >> 6) * kAtomBytes + ptx::sw128_offset(r, n & 63);
                    *reinterpret_cast<uint32_t *>(A2 + off) = w;
                    if (prm.z_out && in && frame < prm.T)
                        prm.z_out[(size_t)frame * prm.K + (n >> 1)] = make_float2(zr, zi);
                }
            }
            // zero the K padding of the GEMM2 A operand
            for (int n = n1; n < prm.k2_atoms * kAtomElems; n += 2) {
                const uint32_t off = (n >> 6) * kAtomBytes + ptx::sw128_offset(r, n & 63);
                *reinterpret_cast<uint32_t *>(A2 + off) = 0u;
            }
            ptx::fence_proxy_async_smem();
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();

    // =============================================================== GEMM2 + top-8
    float tv[kTop];
    int ti[kTop];
#pragma unroll
    for (int i = 0; i < kTop; ++i) {
        tv[i] = -__int_as_float(0x7f800000);
        ti[i] = -1;
    }
    const bool scan = prm.do_scan && !*abort_flag;
    if (scan) {
        if (warp == 8) {
            if (lane == 0) {
                int issued = -1;
                for (int j = 0; j < prm.nq; ++j) {
                    const int u = j & 1;
                    const uint32_t par = ((j >> 1) & 1) ^ 1;
                    if (*abort_flag) break;
                    if (!ptx::mbar_wait(&b2_empty[u], par, budget)) {
                        give_up();
                        break;
                    }
                    ptx::mbar_arrive_expect_tx(&b2_full[u], (uint32_t)(prm.k2_atoms * kAtomBytes));
                    uint8_t *B2 = smem + off_b2 + u * prm.k2_atoms * kAtomBytes;
                    for (int a = 0; a < prm.k2_atoms; ++a)
                        ptx::tma_load_2d(B2 + a * kAtomBytes, &tmap_d, &b2_full[u], a * kAtomElems, j * 128);
                    issued = j;
                }
                for (int j = max(0, issued - 1); j <= issued; ++j)
                    ptx::mbar_wait(&b2_full[j & 1], (j >> 1) & 1, kDrainBudget);
            }
            __syncwarp();
        } else if (warp == 9) {
            if (lane == 0) {
                const uint32_t idesc = ptx::idesc_f16(128, 128, BF16);
                const int steps = prm.k2 >> 4;
                bool ok = true;
                for (int j = 0; j < prm.nq; ++j) {
                    const int u = j & 1;
                    const uint32_t par = (j >> 1) & 1;
                    if (*abort_flag) { ok = false; break; }
                    if (!ptx::mbar_wait(&b2_full[u], par, budget) || !ptx::mbar_wait(&t2_empty[u], par ^ 1, budget)) {
                        give_up();
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint32_t a_base = ptx::smem_u32(smem);
                    const uint32_t b_base = ptx::smem_u32(smem + off_b2 + u * prm.k2_atoms * kAtomBytes);
                    for (int k = 0; k < steps; ++k) {
                        const uint32_t o = (k >> 2) * kAtomBytes + (k & 3) * 32;
                        ptx::mma_f16(tmem + kTmemY + u * 128, ptx::sw128_desc(a_base + o), ptx::sw128_desc(b_base + o),
                                     idesc, k > 0 ? 1u : 0u);
                    }
                    ptx::mma_commit(&b2_empty[u]);
                    ptx::mma_commit(&t2_full[u]);
                }
                (void)ok;
            }
            __syncwarp();
        } else if (warp < 4) {
            for (int j = 0; j < prm.nq; ++j) {
                const int u = j & 1;
                const uint32_t par = (j >> 1) & 1;
                if (*abort_flag) break;
                if (!ptx::mbar_wait(&t2_full[u], par, budget)) {
                    give_up();
                    break;
                }
                ptx::tc_fence_after();
#pragma unroll 1
                for (int c0 = 0; c0 < 128; c0 += 32) {
                    float v[32];
                    ptx::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(kTmemY + u * 128 + c0), v);
                    const int qb = j * 128 + c0;
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const float y = v[i];
                        if (y > tv[kTop - 1] && qb + i < prm.Q) {
                            tv[kTop - 1] = y;
                            ti[kTop - 1] = qb + i;
#pragma unroll
                            for (int x = kTop - 1; x > 0; --x) {
                                if (tv[x] > tv[x - 1]) {
                                    const float fv = tv[x]; tv[x] = tv[x - 1]; tv[x - 1] = fv;
                                    const int iv = ti[x]; ti[x] = ti[x - 1]; ti[x - 1] = iv;
                                }
                            }
                        }
                    }
                }
                ptx::tc_fence_before();
                ptx::mbar_arrive(&t2_empty[u]);
            }
        }
    }
    __syncthreads();

    // =============================================================== rescoring
    if (scan && warp < 4 && !*abort_flag) {
        const int r = tid;
        const long long frame = t0 + r;
        if (frame < prm.T) {
            float best = 0.f;
            int bq = -1;
#pragma unroll
            for (int c = 0; c < kTop; ++c) {
                const int q = ti[c];
                if (q < 0) continue;
                const float2 *dq = prm.Dc32 + (size_t)q * prm.K;
                float acc = 0.f;
                for (int k = 0; k < prm.K; ++k) {
                    const float2 d = __ldg(dq + k);
                    acc = fmaf(d.x, Zf[r * zstride + 2 * k], acc);
                    acc = fmaf(-d.y, Zf[r * zstride + 2 * k + 1], acc);
                }
                if (bq < 0 || acc > best || (acc == best && q < bq)) {
                    best = acc;
                    bq = q;
                }
            }
            prm.idx[frame] = bq;
            if (prm.proj) prm.proj[frame] = bq < 0 ? __int_as_float(0x7fc00000) : best;
        }
    }

    if (warp == 9 && lane == 0 && !drained) {
        ptx::mma_commit(drain);  // completes once every MMA this thread issued is done
        ptx::mbar_wait(drain, 0, kDrainBudget);
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 9) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, kTmemCols);
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

static int encode_2d(CUtensorMap *map, void *base, int bf16, uint64_t inner, uint64_t rows,
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

struct TcMaps {
    CUtensorMap v[2], d[2];
};

int tc_prepare(sp_basis *b) {
    const sp_steering *st = b->st;
    const int K = b->K, P = st->P, B = st->B, Q = st->Q, L = st->L;
    TcLayout t = make_tc_layout(P, B, K);
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
    const int dcols = t.k2_atoms * kAtomElems;
    std::vector<float> df((size_t)Q * dcols, 0.f);
    for (int q = 0; q < Q; ++q)
        for (int kk = 0; kk < K; ++kk) {
            df[(size_t)q * dcols + 2 * kk] = (float)b->D[((size_t)q * K + kk) * 2];
            df[(size_t)q * dcols + 2 * kk + 1] = (float)-b->D[((size_t)q * K + kk) * 2 + 1];
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
        int rc = encode_2d(&maps->v[prec], b->Vtc[prec].p, prec, t.row_elems, t.n1, kAtomElems, t.n1);
        if (rc == SP_OK) rc = encode_2d(&maps->d[prec], b->Dtc[prec].p, prec, dcols, Q, kAtomElems, 128);
        if (rc != SP_OK) {
            delete maps;
            return rc;
        }
    }
    b->tc_maps = maps;
    return SP_OK;
}

void tc_release(sp_basis *b) {
    delete reinterpret_cast<TcMaps *>(b->tc_maps);
    b->tc_maps = nullptr;
}

int launch_svd_tc(const sp_basis *b, const void *frames, int T, int prec, int32_t *idx, float *proj,
                  void *z_out, cudaStream_t s) {
    if (T == 0) return SP_OK;
    const TcLayout &t = b->tc;
    SP_CHECK(t.n1 > 0 && b->tc_maps, SP_ENOTIMPL,
             "tensor-core path supports 2K <= 144 and M <= 16 (use SP_PREC_FP32)");
    const int bf = prec == SP_PREC_BF16 ? 1 : 0;
    const TcMaps *maps = reinterpret_cast<const TcMaps *>(b->tc_maps);
    const SmemPlan plan = make_plan(t);
    TcParams p;
    p.frames = (const float2 *)frames;
    p.T = T;
    p.M = b->st->M;
    p.B = b->st->B;
    p.P = b->st->P;
    p.G = (p.P + kGroupPairs - 1) / kGroupPairs;
    p.n_chunks = t.n_chunks;
    p.n1 = t.n1;
    p.K = b->K;
    p.Q = b->st->Q;
    p.k2 = t.k2;
    p.k2_atoms = t.k2_atoms;
    p.nq = (p.Q + 127) / 128;
    p.inv_vscale = 1.f / b->v_scale;
    p.do_scan = idx != nullptr;
    p.Dc32 = b->Dc32.as<float2>();
    p.idx = idx;
    p.proj = proj;
    p.z_out = (float2 *)z_out;
    static bool attr_set[2] = {false, false};
    if (bf) {
        if (!attr_set[1]) {
            SP_CUDA(cudaFuncSetAttribute(svd_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448));
            attr_set[1] = true;
        }
    } else if (!attr_set[0]) {
        SP_CUDA(cudaFuncSetAttribute(svd_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448));
        attr_set[0] = true;
    }
    SP_CHECK(plan.total <= 232448, SP_ENOTIMPL, "shared-memory plan exceeds 227 KB");
    const unsigned grid = (unsigned)(((long long)T + 127) / 128);
    if (bf)
        svd_tc_kernel<1><<<grid, kThreads, plan.total, s>>>(maps->v[1], maps->d[1], p);
    else
        svd_tc_kernel<0><<<grid, kThreads, plan.total, s>>>(maps->v[0], maps->d[0], p);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

}  // namespace sp

extern "C" int sp_set_wait_budget(long long cycles) {
    using namespace sp;
    const long long v = cycles <= 0 ? 2000000000LL : cycles;
    SP_CUDA(cudaMemcpyToSymbol(g_wait_budget, &v, sizeof(v)));
    h_wait_budget = v;
    return SP_OK;
}
