// Learned direction proposal: a small network proposes coarse cells of the direction grid
// and Eq. 14 is evaluated only over their children, with an exhaustive fallback.  The
// paper has no learned component; the search it narrows is the exhaustive argmax of
// Eq. 14 (Section 3), which stays the judge of every proposed candidate.
//
//   cells      every direction q of the grid belongs to the cell direction with the largest
//              dot product (values within 1e-12 of the largest tie -> lowest cell index);
//   features   x = [Re Z_0, Im Z_0, Re Z_1, ...] / ||Z|| (Z of Eq. 12; x = 0 if ||Z|| = 0);
//   network    h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), logits = W3 h2 + b3;
//   search     children of the n_top cells with the largest logits, argmax Re{D_q Z} in FP32
//              over them; frames whose largest softmax probability is not >= theta take the
//              exhaustive tensor-core scan instead;
//   training   mean softmax cross-entropy against the cell of the frame's exhaustive argmax,
//              Adam (Kingma & Ba, 2015), FP32 master weights.
//
// Kernels: mlp_tc_kernel (inference: the three layers as tcgen05 BF16 GEMMs, FP32 in TMEM,
// bias + ReLU + online softmax + top-8 in the epilogues; activations never leave shared
// memory), rescore_kernel (FP32 Re{D_q Z} over the proposed children), and the training
// kernels (tiled FP32 SIMT GEMMs, softmax cross-entropy, Adam).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "common.h"
#include "ptx.cuh"

namespace sp {
namespace {

constexpr int kMlpThreads = 192;      // warps 0-3: one frame row each thread; 4: TMA; 5: MMA
constexpr int kWRing = 4;             // weight atoms in flight
constexpr int kWAtomBytes = 256 * 128;
constexpr int kAAtomBytes = 128 * 128;
constexpr int kTop = 8;               // cells tracked per frame
constexpr int kMaxF = 320, kMaxH = 256, kMaxC = 4096;
constexpr int kAAtoms = kMaxF / 64;   // A buffer: features (up to 5 atoms) or a hidden layer (4)
constexpr double kCellTie = 1e-12;
constexpr long long kDrain = 4000000000LL;

struct MlpParams {
    const float2 *Z;     // [T][K] complex64
    const float *zn2;    // [T] ||Z||^2
    int T, K, F_atoms, H1, H2, C, n_chunks3, n_tiles;
    const float *b1, *b2, *b3;
    float *logits;       // [T][C] or null
    int32_t *top;        // [T][kTop]
    float *conf;         // [T] largest softmax probability
    int *status;
    long long budget;
};

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// One CTA per SM, tiles of 128 frames.  Per tile the weight atoms (64 input columns of a
// layer's weight rows, <= 256 rows, 128-byte swizzle) stream through a 4-slot TMA ring in
// the order layer 1, layer 2, layer 3 chunk 0, 1, ... (256 cells a chunk).  Accumulators
// alternate between two 256-column TMEM buffers; the 128 row threads turn each finished
// layer into the next layer's A operand (bias, ReLU, BF16) in shared memory, and the last
// layer's chunks into the online softmax and the top-8 cells.
__global__ void __launch_bounds__(kMlpThreads, 1)
    mlp_tc_kernel(const __grid_constant__ CUtensorMap tm1, const __grid_constant__ CUtensorMap tm2,
                  const __grid_constant__ CUtensorMap tm3, const MlpParams prm) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int off_w = kAAtoms * kAAtomBytes;
    const int off_bias = off_w + kWRing * kWAtomBytes;
    const int n_bias = prm.H1 + prm.H2 + prm.C;
    const int off_bar = off_bias + ((n_bias * 4 + 15) / 16) * 16;
    float *bias = reinterpret_cast<float *>(smem + off_bias);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + off_bar);
    uint64_t *w_full = bars, *w_empty = bars + kWRing, *acc_full = bars + 2 * kWRing, *acc_empty = acc_full + 2;
    uint64_t *a_full = acc_empty + 2, *drain = a_full + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(drain + 2);
    const long long budget = prm.budget;

    if (tid == 0) {
        for (int i = 0; i < kWRing; ++i) {
            ptx::mbar_init(&w_full[i], 1);
            ptx::mbar_init(&w_empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(&acc_full[i], 1);
            ptx::mbar_init(&acc_empty[i], 128);
        }
        ptx::mbar_init(a_full, 128);
        ptx::mbar_init(drain, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    for (int i = tid; i < n_bias; i += kMlpThreads)
        bias[i] = i < prm.H1 ? prm.b1[i] : i < prm.H1 + prm.H2 ? prm.b2[i - prm.H1] : prm.b3[i - prm.H1 - prm.H2];
    if (warp == 4 && lane == 0) {
        ptx::prefetch_tmap(&tm1);
        ptx::prefetch_tmap(&tm2);
        ptx::prefetch_tmap(&tm3);
    }
    if (warp == 5) {
        ptx::tmem_alloc(tmem_slot, 512);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int my_tiles = prm.n_tiles > (int)blockIdx.x ? (prm.n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int a1 = prm.F_atoms, a2 = prm.H1 / 64, a3 = prm.H2 / 64;
    const int atoms_per_tile = a1 + a2 + prm.n_chunks3 * a3;
    auto give_up = [&]() {
        *abort_flag = 1;
        atomicOr(prm.status, 2);
    };

    if (warp < 4) {
        // ---------------- row threads: features, hidden layers, logits
        const int r = tid;
        const float *b1 = bias, *b2 = bias + prm.H1, *b3 = bias + prm.H1 + prm.H2;
        uint32_t e_use[2] = {0, 0};
        const uint32_t lane_addr = (uint32_t)(warp * 32) << 16;
        for (int lt = 0; lt < my_tiles && !ptx::warp_flag(abort_flag); ++lt) {
            const long long frame = ((long long)blockIdx.x + (long long)lt * gridDim.x) * 128 + r;
            const bool live = frame < prm.T;
            {   // features x = Z / ||Z|| as BF16 pairs (Re, Im), zero-padded to F_atoms * 64: each
                // warp fills its 32 rows, a row's Z read coalesced by the warp, 4 rows in flight
                const int F2 = prm.F_atoms * 32;
                const long long base = ((long long)blockIdx.x + (long long)lt * gridDim.x) * 128;
                for (int r0 = 0; r0 < 32; r0 += 4) {
                    float2 zv[4][kAAtoms];
                    float inv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const long long fr = base + warp * 32 + r0 + u;
                        const bool lv = fr < prm.T;
                        const float n2 = lv ? prm.zn2[fr] : 0.f;
                        inv[u] = n2 > 0.f ? rsqrtf(n2) : 0.f;
#pragma unroll
                        for (int i = 0; i < kAAtoms; ++i) {
                            const int k = lane + 32 * i;
                            zv[u][i] = (lv && k < prm.K) ? __ldg(prm.Z + (size_t)fr * prm.K + k) : make_float2(0.f, 0.f);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int row = warp * 32 + r0 + u;
#pragma unroll
                        for (int i = 0; i < kAAtoms; ++i) {
                            const int k = lane + 32 * i;
                            if (k < F2) {
                                const int n = 2 * k;
                                *reinterpret_cast<uint32_t *>(smem + (n >> 6) * kAAtomBytes + ptx::sw128_offset(row, n & 63)) =
                                    pack_bf16(zv[u][i].x * inv[u], zv[u][i].y * inv[u]);
                            }
                        }
                    }
                }
                __syncwarp();
            }
            ptx::fence_proxy_async_smem();
            ptx::mbar_arrive(a_full);
            // hidden layers: TMEM buffer 0 (layer 1), then 1 (layer 2)
            for (int layer = 0; layer < 2; ++layer) {
                const int H = layer == 0 ? prm.H1 : prm.H2;
                const float *bb = layer == 0 ? b1 : b2;
                if (!ptx::mbar_wait_warp(&acc_full[layer], e_use[layer] & 1, budget)) {
                    if (lane == 0) give_up();
                    break;
                }
                ++e_use[layer];
                ptx::tc_fence_after();
                for (int cb = 0; cb < H / 64; ++cb) {
                    float v[64];
                    ptx::tmem_ld64(tmem + lane_addr + (uint32_t)(layer * 256 + cb * 64), v);
#pragma unroll
                    for (int i = 0; i < 64; i += 2) {
                        const float h0 = fmaxf(v[i] + bb[cb * 64 + i], 0.f);
                        const float h1 = fmaxf(v[i + 1] + bb[cb * 64 + i + 1], 0.f);
                        *reinterpret_cast<uint32_t *>(smem + cb * kAAtomBytes + ptx::sw128_offset(r, i)) =
                            pack_bf16(h0, h1);
                    }
                }
                ptx::tc_fence_before();
                ptx::mbar_arrive(&acc_empty[layer]);
                ptx::fence_proxy_async_smem();
                ptx::mbar_arrive(a_full);
            }
            if (ptx::warp_flag(abort_flag)) break;
            // output layer in chunks of 256 cells: online softmax and the top-8 cells
            float m = -__int_as_float(0x7f800000), ssum = 0.f;
            float tv[kTop];
            int ti[kTop];
#pragma unroll
            for (int s = 0; s < kTop; ++s) {
                tv[s] = -__int_as_float(0x7f800000);
                ti[s] = -1;
            }
            bool ok = true;
            for (int c = 0; c < prm.n_chunks3; ++c) {
                const int buf = c & 1;
                if (!ptx::mbar_wait_warp(&acc_full[buf], e_use[buf] & 1, budget)) {
                    if (lane == 0) give_up();
                    ok = false;
                    break;
                }
                ++e_use[buf];
                ptx::tc_fence_after();
                for (int cb = 0; cb < 4; ++cb) {
                    float v[64];
                    ptx::tmem_ld64(tmem + lane_addr + (uint32_t)(buf * 256 + cb * 64), v);
                    const int col0 = c * 256 + cb * 64;
                    const float ninf = -__int_as_float(0x7f800000);
#pragma unroll
                    for (int i = 0; i < 64; ++i) v[i] = col0 + i < prm.C ? v[i] + b3[col0 + i] : ninf;
                    if (prm.logits && live) {
#pragma unroll
                        for (int i = 0; i < 64; ++i)
                            if (col0 + i < prm.C) prm.logits[(size_t)frame * prm.C + col0 + i] = v[i];
                    }
                    // online softmax, one chunk of 64 at a time: the chunk maximum by a tree,
                    // then the exponentials in four independent sums
                    float t[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i) t[i] = fmaxf(v[i], v[i + 32]);
#pragma unroll
                    for (int w = 16; w >= 1; w >>= 1)
#pragma unroll
                        for (int i = 0; i < w; ++i) t[i] = fmaxf(t[i], t[i + w]);
                    const float nm = fmaxf(m, t[0]);
                    if (nm > ninf) {
                        float s4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                        for (int i = 0; i < 64; ++i) s4[i & 3] += __expf(v[i] - nm);
                        ssum = ssum * __expf(m - nm) + ((s4[0] + s4[1]) + (s4[2] + s4[3]));
                        m = nm;
                    }
                    // top 8: only values above a threshold go through the (out-of-line) insertion.
                    // The threshold is the 8th best so far; before 8 values have been seen, the
                    // smallest of the 8 group maxima of this chunk (a lower bound of its 8th
                    // largest value), so that about 8 values, not 64, are inserted.
                    float thr = tv[kTop - 1];
                    if (!(thr > ninf)) {
                        float gmin = __int_as_float(0x7f800000);
#pragma unroll
                        for (int g2 = 0; g2 < 8; ++g2) {
                            float gm = v[8 * g2];
#pragma unroll
                            for (int e2 = 1; e2 < 8; ++e2) gm = fmaxf(gm, v[8 * g2 + e2]);
                            gmin = fminf(gmin, gm);
                        }
                        thr = gmin > ninf ? nextafterf(gmin, ninf) : ninf;
                    }
                    unsigned long long hits = 0ull;
#pragma unroll
                    for (int i = 0; i < 64; ++i) hits |= (unsigned long long)(v[i] > thr ? 1u : 0u) << i;
                    while (hits) {
                        const int i = __ffsll((long long)hits) - 1;
                        hits &= hits - 1;
                        float cv = v[0];
#pragma unroll
                        for (int j = 1; j < 64; ++j) cv = i == j ? v[j] : cv;
                        int ci = col0 + i;
#pragma unroll
                        for (int s2 = 0; s2 < kTop; ++s2) {
                            if (cv > tv[s2]) {
                                const float t1 = tv[s2];
                                const int t2 = ti[s2];
                                tv[s2] = cv;
                                ti[s2] = ci;
                                cv = t1;
                                ci = t2;
                            }
                        }
                    }
                }
                ptx::tc_fence_before();
                ptx::mbar_arrive(&acc_empty[buf]);
            }
            if (!ok) break;
            if (live) {
#pragma unroll
                for (int s = 0; s < kTop; ++s) prm.top[(size_t)frame * kTop + s] = ti[s];
                prm.conf[frame] = 1.f / ssum;
            }
        }
    } else if (warp == 4) {
        // ---------------- TMA producer of the weight atoms
        if (lane == 0) {
            long long j = 0, issued = -1;
            for (int lt = 0; lt < my_tiles; ++lt) {
                for (int a = 0; a < atoms_per_tile; ++a, ++j) {
                    if (*abort_flag) break;
                    const int u = (int)(j % kWRing);
                    if (!ptx::mbar_wait(&w_empty[u], (uint32_t)((j / kWRing) & 1) ^ 1u, budget)) {
                        give_up();
                        break;
                    }
                    uint8_t *dst = smem + off_w + u * kWAtomBytes;
                    if (a < a1) {
                        ptx::mbar_arrive_expect_tx(&w_full[u], (uint32_t)prm.H1 * 128u);
                        ptx::tma_load_2d(dst, &tm1, &w_full[u], a * 64, 0);
                    } else if (a < a1 + a2) {
                        ptx::mbar_arrive_expect_tx(&w_full[u], (uint32_t)prm.H2 * 128u);
                        ptx::tma_load_2d(dst, &tm2, &w_full[u], (a - a1) * 64, 0);
                    } else {
                        const int x = a - a1 - a2;
                        ptx::mbar_arrive_expect_tx(&w_full[u], 256u * 128u);
                        ptx::tma_load_2d(dst, &tm3, &w_full[u], (x % a3) * 64, (x / a3) * 256);
                    }
                    issued = j;
                }
                if (*abort_flag) break;
            }
            for (long long q = std::max(0LL, issued - kWRing + 1); q <= issued; ++q)
                ptx::mbar_wait(&w_full[q % kWRing], (uint32_t)((q / kWRing) & 1), kDrain);
        }
        __syncwarp();
    } else {
        // ---------------- MMA issuer
        if (lane == 0) {
            long long j = 0;
            uint32_t a_use = 0, m_use[2] = {0, 0};
            const uint32_t a_base = ptx::smem_u32(smem);
            bool ok = true;
            for (int lt = 0; lt < my_tiles && ok; ++lt) {
                const int n_jobs = 2 + prm.n_chunks3;
                for (int job = 0; job < n_jobs && ok; ++job) {
                    const int buf = job < 2 ? job : (job - 2) & 1;
                    const int n_atoms = job == 0 ? a1 : job == 1 ? a2 : a3;
                    const int N = job == 0 ? prm.H1 : job == 1 ? prm.H2 : 256;
                    const uint32_t idesc = ptx::idesc_f16(128, N, 1);
                    if (job <= 2) {   // a new A operand: features, h1, h2
                        if (*abort_flag || !ptx::mbar_wait(a_full, a_use & 1, budget)) {
                            give_up();
                            ok = false;
                            break;
                        }
                        ++a_use;
                    }
                    if (*abort_flag || !ptx::mbar_wait(&acc_empty[buf], (m_use[buf] & 1) ^ 1u, budget)) {
                        give_up();
                        ok = false;
                        break;
                    }
                    ++m_use[buf];
                    ptx::tc_fence_after();
                    for (int a = 0; a < n_atoms; ++a, ++j) {
                        const int u = (int)(j % kWRing);
                        if (*abort_flag || !ptx::mbar_wait(&w_full[u], (uint32_t)((j / kWRing) & 1), budget)) {
                            give_up();
                            ok = false;
                            break;
                        }
                        ptx::tc_fence_after();
                        const uint32_t b_base = ptx::smem_u32(smem + off_w + u * kWAtomBytes);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            ptx::mma_f16(tmem + (uint32_t)(buf * 256), ptx::sw128_desc(a_base + a * kAAtomBytes + kk * 32),
                                         ptx::sw128_desc(b_base + kk * 32), idesc, (a > 0 || kk > 0) ? 1u : 0u);
                        ptx::mma_commit(&w_empty[u]);
                    }
                    if (!ok) break;
                    ptx::mma_commit(&acc_full[buf]);
                }
            }
            ptx::mma_commit(drain);
            ptx::mbar_wait(drain, 0, kDrain);
        }
        __syncwarp();
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 5) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, 512);
    }
}

// Re{D_q Z} over the children of the proposed cells, one warp per frame.  Screening: the warp
// takes four candidates at a time, eight lanes per candidate row of an FP16 copy of D (rows
// padded to 16-byte multiples), so a load instruction touches four 128-byte lines instead of
// 32; Z sits in shared memory.  A screened score differs from the FP32 one by at most
// e = (2^-11 sqrt(L) + 2^-24 sqrt(K)) ||Z|| (relative FP16 rounding of D, with
// sum_k |D_qk| |Z_k| <= ||D_q|| ||Z|| <= sqrt(L) ||Z||, plus the FP16 subnormal spacing), so
// every candidate whose screened score is within 2e (+ FP32 slack) of the best is rescored
// in FP32 and the best of those is the frame's direction: the result equals an FP32 search
// over all the candidates.  Screened scores and directions wait in shared memory.
constexpr int kMaxCand = 512;     // candidates per frame
constexpr int kMaxKp = 160;       // K <= 160

struct RescoreParams {
    const int32_t *top;
    const float *conf;
    float theta;
    int n_top, T, K, Kp;
    float tol_z, tol_abs;
    const int32_t *cell_ptr, *child, *rep_of;
    const float2 *D;     // [Q][K] FP32
    const uint4 *Dh;     // [Q][Kp] FP16 (Re, Im), Kp = K rounded up to 4
    const float2 *Z;
    int32_t *idx;
    float *proj;
    int32_t *fb_flag;    // [T] or null
    int32_t *fb_list;    // frames that fall back (to the exhaustive tensor-core scan)
    int *fb_count;
};

// FP16 screening of a frame's candidates (directions cq[0 .. total)): candidates c0 + 4h + g,
// h < NR, on lanes 8g .. 8g + 7 (NR rows in flight per group); lane p of a group takes the
// 16-byte pieces p, p + 8, ... (NU of them) of a row.  Scores go to sc[c]; returns the maximum.
template <int NR, int NU>
__device__ __forceinline__ float screen_fp16(const uint4 *__restrict__ Dh, int n16, int Kp, const int *cq, float *sc,
                                             int total, const float2 *z, int lane) {
    const int g = lane >> 3, pl = lane & 7;
    float m = -__int_as_float(0x7f800000);
    for (int c0 = 0; c0 < total; c0 += 4 * NR) {
        int qq[NR];
        uint4 v[NR][NU];
#pragma unroll
        for (int h = 0; h < NR; ++h) {
            const int c = c0 + 4 * h + g;
            qq[h] = c < total ? cq[c] : -1;
            const uint4 *row = Dh + (size_t)(qq[h] >= 0 ? qq[h] : 0) * n16;
#pragma unroll
            for (int u = 0; u < NU; ++u)
                v[h][u] = (qq[h] >= 0 && pl + 8 * u < n16) ? __ldg(row + pl + 8 * u) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int h = 0; h < NR; ++h) {
            float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
            for (int u = 0; u < NU; ++u) {
                const uint32_t wv[4] = {v[h][u].x, v[h][u].y, v[h][u].z, v[h][u].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int k = (pl + 8 * u) * 4 + e;
                    if (k < Kp) {
                        const float2 d = __half22float2(*reinterpret_cast<const __half2 *>(&wv[e]));
                        const float2 zz = z[k];
                        acc0 = fmaf(d.x, zz.x, acc0);
                        acc1 = fmaf(-d.y, zz.y, acc1);
                    }
                }
            }
            float s = acc0 + acc1;
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            s += __shfl_xor_sync(0xffffffffu, s, 2);
            s += __shfl_xor_sync(0xffffffffu, s, 4);
            if (qq[h] >= 0) {
                m = fmaxf(m, s);
                if (pl == 0) sc[c0 + 4 * h + g] = s;
            }
        }
    }
    return m;
}

__global__ void __launch_bounds__(256, 3) rescore_kernel(const RescoreParams prm) {
    __shared__ float2 zs[8][kMaxKp];
    __shared__ float sc_s[8][kMaxCand];
    __shared__ int cq_s[8][kMaxCand];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long frame = (long long)blockIdx.x * 8 + w;
    if (frame >= prm.T) return;   // whole warp
    const int K = prm.K, Kp = prm.Kp;
    const float cf = prm.conf[frame];
    const int32_t *tp = prm.top + (size_t)frame * kTop;
    int lo[kTop], cnt[kTop], total = 0;
#pragma unroll
    for (int t = 0; t < kTop; ++t) {
        const int cell = t < prm.n_top ? tp[t] : -1;
        lo[t] = cell >= 0 ? prm.cell_ptr[cell] : 0;
        cnt[t] = cell >= 0 ? prm.cell_ptr[cell + 1] - lo[t] : 0;
        total += cnt[t];
    }
    if (!(cf >= prm.theta) || tp[0] < 0 || total == 0 || total > kMaxCand) {
        if (lane == 0) {
            prm.fb_list[atomicAdd(prm.fb_count, 1)] = (int32_t)frame;
            if (prm.fb_flag) prm.fb_flag[frame] = 1;
        }
        return;
    }
    float zn2 = 0.f;
    for (int k = lane; k < Kp; k += 32) {
        const float2 z = k < K ? prm.Z[(size_t)frame * K + k] : make_float2(0.f, 0.f);
        zs[w][k] = z;
        zn2 = fmaf(z.x, z.x, fmaf(z.y, z.y, zn2));
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) zn2 += __shfl_xor_sync(0xffffffffu, zn2, o);
    __syncwarp();
    const float2 *z = zs[w];
    // ---- the candidate directions of the frame into shared memory (all loads in flight)
    for (int c = lane; c < total; c += 32) {
        int q = -1, pos = c;
#pragma unroll
        for (int t = 0; t < kTop; ++t) {
            if (q < 0 && pos < cnt[t]) q = prm.child[lo[t] + pos];
            else if (q < 0) pos -= cnt[t];
        }
        cq_s[w][c] = q;
    }
    __syncwarp();
    // ---- screening in FP16
    const int n16 = Kp / 4;   // 16-byte pieces per row (<= 40)
    float m = n16 <= 24 ? screen_fp16<4, 3>(prm.Dh, n16, Kp, cq_s[w], sc_s[w], total, z, lane)
                        : screen_fp16<2, 5>(prm.Dh, n16, Kp, cq_s[w], sc_s[w], total, z, lane);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __syncwarp();
    const float thr = m - (prm.tol_z * sqrtf(zn2) + prm.tol_abs);
    // ---- FP32 rescoring of every candidate in the window, one at a time by the whole warp
    // (lanes over k, coalesced row reads); every lane ends with the same best
    float best = 0.f;
    int bq = -1;
    for (int c0 = 0; c0 < total; c0 += 32) {
        const int c = c0 + lane;
        unsigned sel = __ballot_sync(0xffffffffu, c < total && cq_s[w][c] >= 0 && sc_s[w][c] >= thr);
        while (sel) {
            const int j = __ffs(sel) - 1;
            sel &= sel - 1;
            const int q = cq_s[w][c0 + j];
            const float2 *dq = prm.D + (size_t)q * K;
            float acc = 0.f;
            for (int k = lane; k < K; k += 32) {
                const float2 d = __ldg(dq + k), zz = z[k];
                acc = fmaf(d.x, zz.x, acc);
                acc = fmaf(-d.y, zz.y, acc);
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (bq < 0 || acc > best || (acc == best && q < bq)) {
                best = acc;
                bq = q;
            }
        }
    }
    if (lane == 0) {
        prm.idx[frame] = bq < 0 ? -1 : prm.rep_of[bq];
        if (prm.proj) prm.proj[frame] = bq < 0 ? __int_as_float(0x7fc00000) : best;
        if (prm.fb_flag) prm.fb_flag[frame] = 0;
    }
}

// FP32 complex [Q][K] -> FP16 (Re, Im) pairs [Q][Kp], zero-padded
__global__ void to_half2_kernel(const float2 *in, int Q, int K, int Kp, __half2 *out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)Q * Kp) return;
    const int q = (int)(i / Kp), k = (int)(i % Kp);
    const float2 v = k < K ? in[(size_t)q * K + k] : make_float2(0.f, 0.f);
    out[i] = __floats2half2_rn(v.x, v.y);
}

// ---------------------------------------------------------------- training kernels
// C[m][n] = sum_k A(m, k) B(k, n) (+ bias[n]) (relu), A(m, k) = TA ? A[k lda + m] : A[m lda + k],
// B(k, n) = TB ? B[n ldb + k] : B[k ldb + n].  64 x 64 tiles, 16-deep k steps, 4 x 4 per thread.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) sgemm_kernel(int M, int N, int K, const float *__restrict__ A, int lda,
                                                    const float *__restrict__ B, int ldb, float *__restrict__ C,
                                                    int ldc, const float *__restrict__ bias, int relu) {
    __shared__ float As[16][64 + 4];
    __shared__ float Bs[16][64 + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int i = threadIdx.x; i < 64 * 16; i += 256) {
            const int mm = TA ? (i & 63) : (i >> 4), ka = TA ? (i >> 6) : (i & 15);
            const int gm = m0 + mm, gk = k0 + ka;
            As[ka][mm] = (gm < M && gk < K) ? (TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk]) : 0.f;
            const int nn = TB ? (i >> 4) : (i & 63), kb = TB ? (i & 15) : (i >> 6);
            const int gn = n0 + nn, gk2 = k0 + kb;
            Bs[kb][nn] = (gn < N && gk2 < K) ? (TB ? B[(size_t)gn * ldb + gk2] : B[(size_t)gk2 * ldb + gn]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = As[kk][ty * 4 + i];
                b[i] = Bs[kk][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) acc[i][jj] = fmaf(a[i], b[jj], acc[i][jj]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + jj;
            if (gm < M && gn < N) {
                float v = acc[i][jj] + (bias ? bias[gn] : 0.f);
                if (relu) v = fmaxf(v, 0.f);
                C[(size_t)gm * ldc + gn] = v;
            }
        }
}

// softmax cross-entropy per row: g = (softmax - onehot) / n, loss_row = log sum exp - l[y].
// A label outside [0, C) contributes nothing (g = 0, loss 0).
__global__ void xent_kernel(const float *logits, const int32_t *labels, int n, int C, float *g, float *loss_rows) {
    const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= n) return;
    const float *l = logits + (size_t)row * C;
    float *gr = g + (size_t)row * C;
    const int y = labels[row];
    if (y < 0 || y >= C) {
        for (int c = lane; c < C; c += 32) gr[c] = 0.f;
        if (lane == 0) loss_rows[row] = 0.f;
        return;
    }
    float m = -__int_as_float(0x7f800000);
    for (int c = lane; c < C; c += 32) m = fmaxf(m, l[c]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    float s = 0.f;
    for (int c = lane; c < C; c += 32) s += expf(l[c] - m);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const float inv_n = 1.f / (float)n;
    for (int c = lane; c < C; c += 32) gr[c] = (expf(l[c] - m) / s - (c == y ? 1.f : 0.f)) * inv_n;
    if (lane == 0) loss_rows[row] = logf(s) + m - l[y];
}

// mean of n values in a fixed order (one block)
__global__ void mean_kernel(const float *v, int n, float *out) {
    __shared__ float red[256];
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += 256) s += v[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] / (float)n;
}

// out[c] = sum over rows of g[r][c] (sequential over rows: deterministic)
__global__ void colsum_kernel(const float *g, int n, int H, float *out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= H) return;
    float s = 0.f;
    for (int r = 0; r < n; ++r) s += g[(size_t)r * H + c];
    out[c] = s;
}

// g *= (h > 0): the ReLU derivative (h = relu(z) > 0 exactly where z > 0)
__global__ void relu_back_kernel(float *g, const float *h, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !(h[i] > 0.f)) g[i] = 0.f;
}

__global__ void adam_kernel(float *theta, float *m, float *v, const float *g, long long n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

__global__ void gather_rows_kernel(const float *x, const int32_t *lab, const int32_t *rows, int n, int F, float *xo,
                                   int32_t *lo) {
    const int r = blockIdx.x;
    if (r >= n) return;
    const long long src = rows[r];
    for (int c = threadIdx.x; c < F; c += blockDim.x) xo[(size_t)r * F + c] = x[(size_t)src * F + c];
    if (threadIdx.x == 0) lo[r] = lab[src];
}

// x = interleaved (Re Z, Im Z) / ||Z|| (FP32), warp per frame; label = cell of idx
__global__ void features_kernel(const float2 *Z, int T, int K, const int32_t *idx, const int32_t *cell_of, float *x,
                                int32_t *label) {
    const long long t = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (t >= T) return;
    const float2 *z = Z + (size_t)t * K;
    float s = 0.f;
    for (int k = lane; k < K; k += 32) {
        const float2 v = z[k];
        s = fmaf(v.x, v.x, fmaf(v.y, v.y, s));
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const float inv = s > 0.f ? 1.f / sqrtf(s) : 0.f;
    for (int k = lane; k < K; k += 32) {
        const float2 v = z[k];
        x[(size_t)t * 2 * K + 2 * k] = v.x * inv;
        x[(size_t)t * 2 * K + 2 * k + 1] = v.y * inv;
    }
    if (lane == 0 && label) {
        const int q = idx[t];
        label[t] = q >= 0 ? cell_of[q] : -1;
    }
}

// FP32 master weights -> the BF16 GEMM operands (zero padded)
__global__ void to_bf16_kernel(const float *w, int rows, int cols, int rows_p, int cols_p, __nv_bfloat16 *out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)rows_p * cols_p) return;
    const int r = (int)(i / cols_p), c = (int)(i % cols_p);
    out[i] = __float2bfloat16_rn(r < rows && c < cols ? w[(size_t)r * cols + c] : 0.f);
}

uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

}  // namespace
}  // namespace sp

using namespace sp;

struct sp_proposal {
    const sp_basis *b = nullptr;
    int F = 0, F_atoms = 0, H1 = 0, H2 = 0, C = 0, n_chunks3 = 0;
    long long n_params = 0;
    long long oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
    std::vector<int32_t> cell_of;        // [Q]
    sp::DevBuf d_cell_of, d_cell_ptr, d_child, d_rep_of;
    sp::DevBuf dh;                       // D as FP16 [Q][Kp] (Re, Im) for candidate screening
    int Kp = 0;                          // K rounded up to 4 (16-byte rows)
    sp::DevBuf theta, adam_m, adam_v, grad;
    long long adam_t = 0;
    mutable sp::DevBuf wb1, wb2, wb3;    // BF16 operands
    mutable CUtensorMap tm[3];
    mutable bool dirty = true;
    mutable sp::DevBuf work;             // training activations
    mutable sp::DevBuf lwork;            // localisation scratch
};

namespace {

int refresh_bf16(const sp_proposal *p, cudaStream_t s) {
    if (!p->dirty) return SP_OK;
    const int Fp = p->F_atoms * 64, Cp = p->n_chunks3 * 256;
    SP_TRY(p->wb1.reserve((size_t)p->H1 * Fp * 2));
    SP_TRY(p->wb2.reserve((size_t)p->H2 * p->H1 * 2));
    SP_TRY(p->wb3.reserve((size_t)Cp * p->H2 * 2));
    const float *th = p->theta.as<float>();
    auto conv = [&](const float *w, int rows, int cols, int rp, int cp, void *out) -> int {
        const long long n = (long long)rp * cp;
        to_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w, rows, cols, rp, cp,
                                                                    static_cast<__nv_bfloat16 *>(out));
        SP_CUDA(cudaGetLastError());
        return SP_OK;
    };
    SP_TRY(conv(th + p->oW1, p->H1, p->F, p->H1, Fp, p->wb1.p));
    SP_TRY(conv(th + p->oW2, p->H2, p->H1, p->H2, p->H1, p->wb2.p));
    SP_TRY(conv(th + p->oW3, p->C, p->H2, Cp, p->H2, p->wb3.p));
    SP_TRY(encode_tmap_2d(&p->tm[0], p->wb1.p, 1, Fp, p->H1, 64, p->H1));
    SP_TRY(encode_tmap_2d(&p->tm[1], p->wb2.p, 1, p->H1, p->H2, 64, p->H2));
    SP_TRY(encode_tmap_2d(&p->tm[2], p->wb3.p, 1, p->H2, Cp, 64, 256));
    p->dirty = false;
    return SP_OK;
}

int sgemm(bool ta, bool tb, int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *C, int ldc,
          const float *bias, bool relu, cudaStream_t s) {
    if (M == 0 || N == 0) return SP_OK;
    dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64));
    const int r = relu ? 1 : 0;
    if (!ta && !tb) sgemm_kernel<false, false><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, r);
    else if (!ta && tb) sgemm_kernel<false, true><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, r);
    else if (ta && !tb) sgemm_kernel<true, false><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, r);
    else sgemm_kernel<true, true><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, r);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

// FP32 forward of n rows: h1 [n][H1], h2 [n][H2], logits [n][C] in the work buffer.
struct Fwd {
    float *h1, *h2, *logits, *g_logits, *g_h2, *g_h1, *loss_rows, *xb;
    int32_t *lb;
};

int work_for(const sp_proposal *p, int n, Fwd *f) {
    const size_t need = (size_t)n * (2 * (p->H1 + p->H2) + 2 * p->C + 1 + p->F + 1) * 4 + 8 * 256;
    SP_TRY(p->work.reserve(need));
    float *w = p->work.as<float>();
    auto take = [&](size_t cnt) {
        float *r = w;
        w += (cnt + 63) / 64 * 64;
        return r;
    };
    f->h1 = take((size_t)n * p->H1);
    f->h2 = take((size_t)n * p->H2);
    f->logits = take((size_t)n * p->C);
    f->g_logits = take((size_t)n * p->C);
    f->g_h2 = take((size_t)n * p->H2);
    f->g_h1 = take((size_t)n * p->H1);
    f->loss_rows = take((size_t)n);
    f->xb = take((size_t)n * p->F);
    f->lb = reinterpret_cast<int32_t *>(take((size_t)n));
    return SP_OK;
}

int forward_f32(const sp_proposal *p, const float *x, int n, const Fwd &f, cudaStream_t s) {
    const float *th = p->theta.as<float>();
    SP_TRY(sgemm(false, true, n, p->H1, p->F, x, p->F, th + p->oW1, p->F, f.h1, p->H1, th + p->ob1, true, s));
    SP_TRY(sgemm(false, true, n, p->H2, p->H1, f.h1, p->H1, th + p->oW2, p->H1, f.h2, p->H2, th + p->ob2, true, s));
    SP_TRY(sgemm(false, true, n, p->C, p->H2, f.h2, p->H2, th + p->oW3, p->H2, f.logits, p->C, th + p->ob3, false, s));
    return SP_OK;
}

// loss and gradient (parameter layout) of n rows
int backward_f32(const sp_proposal *p, const float *x, const int32_t *lab, int n, const Fwd &f, float *grad,
                 float *loss, cudaStream_t s) {
    const float *th = p->theta.as<float>();
    xent_kernel<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(f.logits, lab, n, p->C, f.g_logits, f.loss_rows);
    SP_CUDA(cudaGetLastError());
    if (loss) {
        mean_kernel<<<1, 256, 0, s>>>(f.loss_rows, n, loss);
        SP_CUDA(cudaGetLastError());
    }
    // output layer
    SP_TRY(sgemm(true, false, p->C, p->H2, n, f.g_logits, p->C, f.h2, p->H2, grad + p->oW3, p->H2, nullptr, false, s));
    colsum_kernel<<<(unsigned)((p->C + 255) / 256), 256, 0, s>>>(f.g_logits, n, p->C, grad + p->ob3);
    SP_TRY(sgemm(false, false, n, p->H2, p->C, f.g_logits, p->C, th + p->oW3, p->H2, f.g_h2, p->H2, nullptr, false, s));
    relu_back_kernel<<<(unsigned)(((long long)n * p->H2 + 255) / 256), 256, 0, s>>>(f.g_h2, f.h2, (long long)n * p->H2);
    // layer 2
    SP_TRY(sgemm(true, false, p->H2, p->H1, n, f.g_h2, p->H2, f.h1, p->H1, grad + p->oW2, p->H1, nullptr, false, s));
    colsum_kernel<<<(unsigned)((p->H2 + 255) / 256), 256, 0, s>>>(f.g_h2, n, p->H2, grad + p->ob2);
    SP_TRY(sgemm(false, false, n, p->H1, p->H2, f.g_h2, p->H2, th + p->oW2, p->H1, f.g_h1, p->H1, nullptr, false, s));
    relu_back_kernel<<<(unsigned)(((long long)n * p->H1 + 255) / 256), 256, 0, s>>>(f.g_h1, f.h1, (long long)n * p->H1);
    // layer 1
    SP_TRY(sgemm(true, false, p->H1, p->F, n, f.g_h1, p->H1, x, p->F, grad + p->oW1, p->F, nullptr, false, s));
    colsum_kernel<<<(unsigned)((p->H1 + 255) / 256), 256, 0, s>>>(f.g_h1, n, p->H1, grad + p->ob1);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

int check_batch(const sp_proposal *p, const void *x, const void *lab, int n) {
    SP_CHECK(p, SP_EINVAL, "proposal: null handle");
    SP_CHECK(n >= 1 && n <= (1 << 20), SP_EINVAL, "proposal: batch size must be in [1, 2^20]");
    SP_CHECK(x, SP_EINVAL, "proposal: null feature pointer");
    (void)lab;
    return SP_OK;
}

int launch_mlp(const sp_proposal *p, const void *Z, const float *zn2, int T, float *logits, int32_t *top, float *conf,
               cudaStream_t s) {
    if (T == 0) return SP_OK;
    SP_TRY(refresh_bf16(p, s));
    MlpParams m;
    m.Z = static_cast<const float2 *>(Z);
    m.zn2 = zn2;
    m.T = T;
    m.K = p->b->K;
    m.F_atoms = p->F_atoms;
    m.H1 = p->H1;
    m.H2 = p->H2;
    m.C = p->C;
    m.n_chunks3 = p->n_chunks3;
    m.n_tiles = (T + 127) / 128;
    const float *th = p->theta.as<float>();
    m.b1 = th + p->ob1;
    m.b2 = th + p->ob2;
    m.b3 = th + p->ob3;
    m.logits = logits;
    m.top = top;
    m.conf = conf;
    SP_TRY(device_status_ptr(&m.status));
    m.budget = wait_budget();
    const int n_bias = p->H1 + p->H2 + p->C;
    const int smem = kAAtoms * kAAtomBytes + kWRing * kWAtomBytes + ((n_bias * 4 + 15) / 16) * 16 +
                     (2 * kWRing + 6) * 8 + 16 + 1024;
    SP_TRY(ensure_max_smem((const void *)mlp_tc_kernel));
    SP_CHECK(smem <= 232448, SP_ENOTIMPL, "proposal: network too large for the shared-memory plan");
    const int grid = std::min(m.n_tiles, num_sms());
    mlp_tc_kernel<<<grid, kMlpThreads, smem, s>>>(p->tm[0], p->tm[1], p->tm[2], m);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

}  // namespace

extern "C" {

int sp_proposal_create(const sp_basis *b, const double *cell_dirs, int C, int H1, int H2, unsigned long long seed,
                       sp_proposal **out) {
    SP_CHECK(out, SP_EINVAL, "sp_proposal_create: out is NULL");
    *out = nullptr;
    SP_CHECK(b && cell_dirs, SP_EINVAL, "sp_proposal_create: null basis or cell directions");
    SP_CHECK(C >= 1 && C <= kMaxC, SP_EINVAL, "sp_proposal_create: C must be in [1, 4096]");
    SP_CHECK(H1 >= 64 && H1 <= kMaxH && H1 % 64 == 0 && H2 >= 64 && H2 <= kMaxH && H2 % 64 == 0, SP_EINVAL,
             "sp_proposal_create: hidden sizes must be multiples of 64 in [64, 256]");
    SP_CHECK(2 * b->K <= kMaxF && b->K <= kMaxKp && b->tc.n1 > 0 && b->tc_maps, SP_ENOTIMPL,
             "sp_proposal_create: the basis needs the tensor-core plan of GEMM1 (2K <= 288, M <= 16)");
    for (int c = 0; c < C; ++c) {
        const double *d = cell_dirs + 3 * c;
        SP_CHECK(std::isfinite(d[0]) && std::isfinite(d[1]) && std::isfinite(d[2]) &&
                     (d[0] != 0 || d[1] != 0 || d[2] != 0),
                 SP_EINVAL, "sp_proposal_create: bad cell direction");
    }
    sp_proposal *p = new (std::nothrow) sp_proposal();
    SP_CHECK(p, SP_ENOMEM, "sp_proposal_create: host allocation failed");
    std::unique_ptr<sp_proposal> guard(p);
    p->b = b;
    p->F = 2 * b->K;
    p->F_atoms = (p->F + 63) / 64;
    p->H1 = H1;
    p->H2 = H2;
    p->C = C;
    p->n_chunks3 = (C + 255) / 256;
    p->oW1 = 0;
    p->ob1 = p->oW1 + (long long)H1 * p->F;
    p->oW2 = p->ob1 + H1;
    p->ob2 = p->oW2 + (long long)H2 * H1;
    p->oW3 = p->ob2 + H2;
    p->ob3 = p->oW3 + (long long)C * H2;
    p->n_params = p->ob3 + C;
    // cells and their children (host, FP64)
    const sp_steering *st = b->st;
    const int Q = st->Q;
    std::vector<double> cn((size_t)C * 3);
    for (int c = 0; c < C; ++c) {
        const double *d = cell_dirs + 3 * c;
        const double n = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int i = 0; i < 3; ++i) cn[3 * c + i] = d[i] / n;
    }
    p->cell_of.resize(Q);
    std::vector<double> dots(C);
    for (int q = 0; q < Q; ++q) {
        const double *f = &st->dirs[3 * (size_t)q];
        const double n = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
        const double fx = f[0] / n, fy = f[1] / n, fz = f[2] / n;
        double best = -2.0;
        for (int c = 0; c < C; ++c) {
            dots[c] = cn[3 * c] * fx + cn[3 * c + 1] * fy + cn[3 * c + 2] * fz;
            best = std::max(best, dots[c]);
        }
        int cell = 0;
        while (dots[cell] < best - kCellTie) ++cell;
        p->cell_of[q] = cell;
    }
    std::vector<int32_t> ptr(C + 1, 0), child(Q);
    for (int q = 0; q < Q; ++q) ++ptr[p->cell_of[q] + 1];
    for (int c = 0; c < C; ++c) ptr[c + 1] += ptr[c];
    {
        std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
        for (int q = 0; q < Q; ++q) child[fill[p->cell_of[q]]++] = q;   // ascending within a cell
    }
    std::vector<int32_t> rep(st->rep_of.begin(), st->rep_of.end());
    SP_TRY(p->d_cell_of.reserve((size_t)Q * 4));
    SP_TRY(p->d_cell_ptr.reserve((size_t)(C + 1) * 4));
    SP_TRY(p->d_child.reserve((size_t)Q * 4));
    SP_TRY(p->d_rep_of.reserve((size_t)Q * 4));
    SP_CUDA(cudaMemcpy(p->d_cell_of.p, p->cell_of.data(), (size_t)Q * 4, cudaMemcpyHostToDevice));
    SP_CUDA(cudaMemcpy(p->d_cell_ptr.p, ptr.data(), (size_t)(C + 1) * 4, cudaMemcpyHostToDevice));
    SP_CUDA(cudaMemcpy(p->d_child.p, child.data(), (size_t)Q * 4, cudaMemcpyHostToDevice));
    SP_CUDA(cudaMemcpy(p->d_rep_of.p, rep.data(), (size_t)Q * 4, cudaMemcpyHostToDevice));
    {
        p->Kp = (b->K + 3) / 4 * 4;
        const long long n = (long long)Q * p->Kp;
        SP_TRY(p->dh.reserve((size_t)n * 4));
        to_half2_kernel<<<(unsigned)((n + 255) / 256), 256>>>(b->Dc32.as<float2>(), Q, b->K, p->Kp,
                                                                p->dh.as<__half2>());
        SP_CUDA(cudaGetLastError());
    }
    // parameters: weights uniform in +-sqrt(6 / fan_in) from a counter-based generator, biases 0
    std::vector<float> th((size_t)p->n_params, 0.f);
    auto init = [&](long long off, int rows, int cols) {
        const double a = std::sqrt(6.0 / cols);
        for (long long i = 0; i < (long long)rows * cols; ++i) {
            const uint64_t u = splitmix64(seed ^ (uint64_t)(off + i) * 0xD1B54A32D192ED03ULL);
            const double r = (double)(u >> 11) * (1.0 / 9007199254740992.0);
            th[(size_t)(off + i)] = (float)((2.0 * r - 1.0) * a);
        }
    };
    init(p->oW1, H1, p->F);
    init(p->oW2, H2, H1);
    init(p->oW3, C, H2);
    SP_TRY(p->theta.reserve((size_t)p->n_params * 4));
    SP_TRY(p->adam_m.reserve((size_t)p->n_params * 4));
    SP_TRY(p->adam_v.reserve((size_t)p->n_params * 4));
    SP_TRY(p->grad.reserve((size_t)p->n_params * 4));
    SP_CUDA(cudaMemcpy(p->theta.p, th.data(), th.size() * 4, cudaMemcpyHostToDevice));
    SP_CUDA(cudaMemset(p->adam_m.p, 0, th.size() * 4));
    SP_CUDA(cudaMemset(p->adam_v.p, 0, th.size() * 4));
    SP_CUDA(cudaDeviceSynchronize());
    *out = guard.release();
    return SP_OK;
}

void sp_proposal_destroy(sp_proposal *p) { delete p; }

int sp_proposal_dims(const sp_proposal *p, int *F, int *H1, int *H2, int *C, long long *n_params) {
    SP_CHECK(p, SP_EINVAL, "sp_proposal_dims: null handle");
    if (F) *F = p->F;
    if (H1) *H1 = p->H1;
    if (H2) *H2 = p->H2;
    if (C) *C = p->C;
    if (n_params) *n_params = p->n_params;
    return SP_OK;
}

int sp_proposal_cells(const sp_proposal *p, int32_t *cell_of_host) {
    SP_CHECK(p && cell_of_host, SP_EINVAL, "sp_proposal_cells: null pointer");
    std::memcpy(cell_of_host, p->cell_of.data(), p->cell_of.size() * 4);
    return SP_OK;
}

int sp_proposal_get_params(const sp_proposal *p, float *host) {
    SP_CHECK(p && host, SP_EINVAL, "sp_proposal_get_params: null pointer");
    SP_CUDA(cudaDeviceSynchronize());
    SP_CUDA(cudaMemcpy(host, p->theta.p, (size_t)p->n_params * 4, cudaMemcpyDeviceToHost));
    return SP_OK;
}

int sp_proposal_set_params(sp_proposal *p, const float *host) {
    SP_CHECK(p && host, SP_EINVAL, "sp_proposal_set_params: null pointer");
    for (long long i = 0; i < p->n_params; ++i)
        SP_CHECK(std::isfinite(host[i]), SP_EINVAL, "sp_proposal_set_params: non-finite parameter");
    SP_CUDA(cudaDeviceSynchronize());
    SP_CUDA(cudaMemcpy(p->theta.p, host, (size_t)p->n_params * 4, cudaMemcpyHostToDevice));
    SP_CUDA(cudaMemset(p->adam_m.p, 0, (size_t)p->n_params * 4));
    SP_CUDA(cudaMemset(p->adam_v.p, 0, (size_t)p->n_params * 4));
    p->adam_t = 0;
    p->dirty = true;
    return SP_OK;
}

int sp_proposal_examples(const sp_proposal *p, const void *frames_dev, int T, sp_prec prec, float *x_dev,
                         int32_t *label_dev, void *stream) {
    SP_CHECK(p, SP_EINVAL, "sp_proposal_examples: null handle");
    SP_CHECK(T >= 0, SP_EINVAL, "sp_proposal_examples: T < 0");
    if (T == 0) return SP_OK;
    SP_CHECK(frames_dev && x_dev && label_dev, SP_EINVAL, "sp_proposal_examples: null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    const int K = p->b->K;
    SP_TRY(p->lwork.reserve((size_t)T * (8 * K + 4)));
    float2 *Z = p->lwork.as<float2>();
    int32_t *idx = reinterpret_cast<int32_t *>(Z + (size_t)T * K);
    SP_TRY(sp_project(p->b, frames_dev, T, prec, Z, stream));
    SP_TRY(sp_localize(p->b, frames_dev, T, SP_MODE_SVD_EXHAUSTIVE, prec, idx, nullptr, nullptr, stream));
    features_kernel<<<(unsigned)((T + 7) / 8), 256, 0, s>>>(Z, T, K, idx, p->d_cell_of.as<int32_t>(), x_dev,
                                                              label_dev);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

int sp_proposal_forward_f32(const sp_proposal *p, const float *x_dev, int n, float *logits_dev, void *stream) {
    SP_TRY(check_batch(p, x_dev, nullptr, n));
    SP_CHECK(logits_dev, SP_EINVAL, "sp_proposal_forward_f32: null logits pointer");
    cudaStream_t s = (cudaStream_t)stream;
    Fwd f;
    SP_TRY(work_for(p, n, &f));
    SP_TRY(forward_f32(p, x_dev, n, f, s));
    SP_CUDA(cudaMemcpyAsync(logits_dev, f.logits, (size_t)n * p->C * 4, cudaMemcpyDeviceToDevice, s));
    return SP_OK;
}

int sp_proposal_grad(const sp_proposal *p, const float *x_dev, const int32_t *label_dev, int n, float *grad_dev,
                     float *loss_dev, void *stream) {
    SP_TRY(check_batch(p, x_dev, label_dev, n));
    SP_CHECK(label_dev && grad_dev, SP_EINVAL, "sp_proposal_grad: null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    Fwd f;
    SP_TRY(work_for(p, n, &f));
    SP_TRY(forward_f32(p, x_dev, n, f, s));
    SP_TRY(backward_f32(p, x_dev, label_dev, n, f, grad_dev, loss_dev, s));
    return SP_OK;
}

int sp_proposal_train_step(sp_proposal *p, const float *x_dev, const int32_t *label_dev, const int32_t *rows_dev,
                           int n, float lr, float *loss_dev, void *stream) {
    SP_TRY(check_batch(p, x_dev, label_dev, n));
    SP_CHECK(label_dev, SP_EINVAL, "sp_proposal_train_step: null label pointer");
    SP_CHECK(lr > 0 && std::isfinite(lr), SP_EINVAL, "sp_proposal_train_step: lr must be positive");
    cudaStream_t s = (cudaStream_t)stream;
    Fwd f;
    SP_TRY(work_for(p, n, &f));
    const float *x = x_dev;
    const int32_t *lab = label_dev;
    if (rows_dev) {
        gather_rows_kernel<<<(unsigned)n, 128, 0, s>>>(x_dev, label_dev, rows_dev, n, p->F, f.xb, f.lb);
        SP_CUDA(cudaGetLastError());
        x = f.xb;
        lab = f.lb;
    }
    SP_TRY(forward_f32(p, x, n, f, s));
    SP_TRY(backward_f32(p, x, lab, n, f, p->grad.as<float>(), loss_dev, s));
    p->adam_t += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 / (1.0 - std::pow(b1, (double)p->adam_t)));
    const float c2 = (float)(1.0 / (1.0 - std::pow(b2, (double)p->adam_t)));
    adam_kernel<<<(unsigned)((p->n_params + 255) / 256), 256, 0, s>>>(
        p->theta.as<float>(), p->adam_m.as<float>(), p->adam_v.as<float>(), p->grad.as<float>(), p->n_params, lr,
        (float)b1, (float)b2, 1e-8f, c1, c2);
    SP_CUDA(cudaGetLastError());
    p->dirty = true;
    return SP_OK;
}

int sp_proposal_infer(const sp_proposal *p, const void *z_dev, const float *zn2_dev, int T, float *logits_dev,
                      int32_t *top_dev, float *conf_dev, void *stream) {
    SP_CHECK(p, SP_EINVAL, "sp_proposal_infer: null handle");
    SP_CHECK(T >= 0, SP_EINVAL, "sp_proposal_infer: T < 0");
    if (T == 0) return SP_OK;
    SP_CHECK(z_dev && zn2_dev && top_dev && conf_dev, SP_EINVAL, "sp_proposal_infer: null pointer");
    return launch_mlp(p, z_dev, zn2_dev, T, logits_dev, top_dev, conf_dev, (cudaStream_t)stream);
}

int sp_localize_learned(const sp_proposal *p, const void *frames_dev, int T, sp_prec prec, int n_top, float theta,
                        int32_t *idx_dev, float *score_dev, float *proj_score_dev, int32_t *fallback_dev,
                        void *stream) {
    SP_CHECK(p, SP_EINVAL, "sp_localize_learned: null handle");
    SP_CHECK(T >= 0, SP_EINVAL, "sp_localize_learned: T < 0");
    SP_CHECK(prec == SP_PREC_FP16 || prec == SP_PREC_BF16, SP_ENOTIMPL,
             "sp_localize_learned: prec must be SP_PREC_FP16 or SP_PREC_BF16");
    SP_CHECK(n_top >= 1 && n_top <= kTop, SP_EINVAL, "sp_localize_learned: n_top must be in [1, 8]");
    SP_CHECK(std::isfinite(theta), SP_EINVAL, "sp_localize_learned: theta must be finite");
    if (T == 0) return SP_OK;
    SP_CHECK(frames_dev && idx_dev, SP_EINVAL, "sp_localize_learned: null frames or idx pointer");
    const sp_basis *b = p->b;
    cudaStream_t s = (cudaStream_t)stream;
    const int K = b->K;
    const size_t zb = ((size_t)T * K * 8 + 255) / 256 * 256;
    const size_t nb = ((size_t)T * 4 + 255) / 256 * 256;
    const size_t sb = (scan_workspace_bytes(T) + 255) / 256 * 256;
    SP_TRY(p->lwork.reserve(zb + nb * (3 + kTop) + sb + 256));
    char *w = p->lwork.as<char>();
    float2 *Z = reinterpret_cast<float2 *>(w);
    float *zn2 = reinterpret_cast<float *>(w + zb);
    float *conf = reinterpret_cast<float *>(w + zb + nb);
    int32_t *fb_list = reinterpret_cast<int32_t *>(w + zb + 2 * nb);
    int32_t *top = reinterpret_cast<int32_t *>(w + zb + 3 * nb);
    void *scan_ws = w + zb + (3 + kTop) * nb;
    int *fb_count = reinterpret_cast<int *>(w + zb + (3 + kTop) * nb + sb);
    SP_TRY(launch_svd_proj(b, frames_dev, T, (int)prec, Z, zn2, s));
    SP_TRY(launch_mlp(p, Z, zn2, T, nullptr, top, conf, s));
    SP_CUDA(cudaMemsetAsync(fb_count, 0, sizeof(int), s));
    RescoreParams r;
    r.top = top;
    r.conf = conf;
    r.theta = theta;
    r.n_top = n_top;
    r.T = T;
    r.K = K;
    r.cell_ptr = p->d_cell_ptr.as<int32_t>();
    r.child = p->d_child.as<int32_t>();
    r.rep_of = p->d_rep_of.as<int32_t>();
    r.D = b->Dc32.as<float2>();
    r.Dh = p->dh.as<uint4>();
    r.Kp = p->Kp;
    r.tol_z = (float)(2.0 * (std::ldexp(1.0, -11) * std::sqrt((double)b->st->L) + std::ldexp(1.0, -24) * std::sqrt((double)K)));
    r.tol_abs = (float)(2.0 * 1e-6 * b->st->L);
    r.Z = Z;
    r.idx = idx_dev;
    r.proj = proj_score_dev;
    r.fb_flag = fallback_dev;
    r.fb_list = fb_list;
    r.fb_count = fb_count;
    rescore_kernel<<<(unsigned)((T + 7) / 8), 256, 0, s>>>(r);
    SP_CUDA(cudaGetLastError());
    // the frames that fell back: the exhaustive tensor-core scan of sp_localize on the listed
    // frames only (CTAs past the device-side count exit at once)
    SP_TRY(launch_svd_scan(b, Z, zn2, T, (int)prec, idx_dev, proj_score_dev, s, scan_ws, fb_list, fb_count));
    if (score_dev) SP_TRY(launch_score_row(b->st, frames_dev, T, idx_dev, score_dev, s));
    return SP_OK;
}

}  // extern "C"
