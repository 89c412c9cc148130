// Offline step 4 and online step 3 of Algorithm 1: a k-d tree (Bentley 1975) over the
// normalised rows D^_q = D_q / ||D_q|| and its exact nearest-neighbour search (Eq. 15).
//
// Eq. 15: Re{D^_q Z^} = 1 - ||D^_q - conj(Z^)||^2 / 2 for unit vectors, so the direction
// maximising the normalised score is the nearest neighbour of conj(Z^) among the D^_q,
// searched in the real 2K-dimensional embedding x_q = [Re D^_q, Im D^_q] with query
// [Re Z^, -Im Z^].
//
// Build (host): one point per direction class (directions with identical TDOA vectors
// have identical rows D_q); split on the dimension of largest spread at the median (ties
// broken by index), recursively, until a node holds at most 32 points (one leaf bucket =
// one warp).
// Search (device): one warp per query; the warp walks the tree with an explicit stack,
// visiting the near child first and keeping the far child only if the squared distance
// from the query to the splitting plane does not exceed the best distance so far
// (exact search).  A leaf's 32 points are stored dimension-major so that lane j reads
// point j coalesced; lanes then reduce (distance, index) to the lexicographic minimum.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "common.h"
#include "debug.cuh"

namespace sp {

constexpr int kLeaf = 32;
constexpr int kMaxDepth = 64;
constexpr int kMaxDims = 512;

namespace {
struct Builder {
    int dim = 0;
    const std::vector<float> *pts = nullptr;   // Q x dim
    std::vector<KdNode> nodes;
    std::vector<int> bucket_ids;                // n_buckets x 32 (-1 = empty slot)
    int depth = 0;

    float x(int id, int d) const { return (*pts)[(size_t)id * dim + d]; }

    int build(std::vector<int> &ids, int lo, int hi, int level) {
        depth = std::max(depth, level + 1);
        const int me = (int)nodes.size();
        nodes.push_back(KdNode{-1, 0.f, 0, 0});
        if (hi - lo <= kLeaf) {
            const int bucket = (int)(bucket_ids.size() / kLeaf);
            for (int i = 0; i < kLeaf; ++i) bucket_ids.push_back(lo + i < hi ? ids[lo + i] : -1);
            nodes[me] = KdNode{-1, 0.f, bucket, hi - lo};
            return me;
        }
        int best_d = 0;
        float best_spread = -1.f;
        for (int d = 0; d < dim; ++d) {
            float mn = x(ids[lo], d), mx = mn;
            for (int i = lo + 1; i < hi; ++i) {
                const float v = x(ids[i], d);
                mn = std::min(mn, v);
                mx = std::max(mx, v);
            }
            if (mx - mn > best_spread) {
                best_spread = mx - mn;
                best_d = d;
            }
        }
        std::sort(ids.begin() + lo, ids.begin() + hi, [&](int a, int b) {
            const float va = x(a, best_d), vb = x(b, best_d);
            return va < vb || (va == vb && a < b);
        });
        const int mid = (lo + hi) / 2;
        const float split = x(ids[mid], best_d);  // left: x <= split, right: x >= split
        build(ids, lo, mid, level + 1);
        const int right = build(ids, mid, hi, level + 1);
        nodes[me] = KdNode{best_d, split, right, 0};
        return me;
    }
};
}  // namespace

int build_kdtree(sp_basis *b) {
    const int Q = b->st->Q, K = b->K, dim = 2 * K;
    SP_CHECK(dim <= kMaxDims, SP_ENOTIMPL, "k-d tree supports 2K <= 512");
    std::vector<float> pts((size_t)Q * dim);
    for (int q = 0; q < Q; ++q) {
        double n2 = 0;
        for (int k = 0; k < K; ++k) {
            const double re = b->D[((size_t)q * K + k) * 2], im = b->D[((size_t)q * K + k) * 2 + 1];
            n2 += re * re + im * im;
        }
        const double inv = n2 > 0 ? 1.0 / std::sqrt(n2) : 0.0;
        for (int k = 0; k < K; ++k) {
            pts[(size_t)q * dim + k] = (float)(b->D[((size_t)q * K + k) * 2] * inv);
            pts[(size_t)q * dim + K + k] = (float)(b->D[((size_t)q * K + k) * 2 + 1] * inv);
        }
    }
    Builder bd;
    bd.dim = dim;
    bd.pts = &pts;
    std::vector<int> ids(b->st->reps);   // one point per direction class (identical rows)
    bd.build(ids, 0, (int)ids.size(), 0);
    SP_CHECK(bd.depth <= kMaxDepth, SP_ENOTIMPL, "k-d tree too deep");
    const int nb = (int)(bd.bucket_ids.size() / kLeaf);
    std::vector<float> leaf((size_t)nb * dim * kLeaf, 1e18f);
    for (int bkt = 0; bkt < nb; ++bkt)
        for (int j = 0; j < kLeaf; ++j) {
            const int id = bd.bucket_ids[(size_t)bkt * kLeaf + j];
            if (id < 0) continue;
            for (int d = 0; d < dim; ++d)
                leaf[((size_t)bkt * dim + d) * kLeaf + j] = pts[(size_t)id * dim + d];
        }
    b->nodes_host = bd.nodes;
    b->n_nodes = (int)bd.nodes.size();
    b->depth = bd.depth;
    b->leaf_size = kLeaf;
    b->n_slots = nb * kLeaf;
    SP_TRY(b->nodes.reserve(bd.nodes.size() * sizeof(KdNode)));
    SP_TRY(b->leaf_pts.reserve(leaf.size() * 4));
    SP_TRY(b->leaf_ids.reserve(bd.bucket_ids.size() * 4));
    SP_CUDA(cudaMemcpy(b->nodes.p, bd.nodes.data(), bd.nodes.size() * sizeof(KdNode), cudaMemcpyHostToDevice));
    SP_CUDA(cudaMemcpy(b->leaf_pts.p, leaf.data(), leaf.size() * 4, cudaMemcpyHostToDevice));
    SP_CUDA(cudaMemcpy(b->leaf_ids.p, bd.bucket_ids.data(), bd.bucket_ids.size() * 4, cudaMemcpyHostToDevice));
    return SP_OK;
}

// One warp per query, KD_WARPS warps per CTA, CTAs striding over the queries.  Shared memory:
// the tree's nodes (when they fit in kNodeSmem bytes; else they are read from global memory),
// then per warp the query (2K floats) and the stack.  visits (optional, int32 [T][2]) receives,
// per query, the nodes and the leaf buckets (32 points each) the search visited.
constexpr int KD_WARPS = 8;
constexpr int kNodeSmem = 96 * 1024;

__global__ void __launch_bounds__(KD_WARPS * 32)
    kdtree_kernel(const float2 *__restrict__ Z, int T, int K, const KdNode *__restrict__ nodes_g, int n_nodes,
                  int nodes_in_smem, const float *__restrict__ leaf_pts, const int32_t *__restrict__ leaf_ids,
                  int32_t *__restrict__ idx_out, float *__restrict__ proj_out, int32_t *__restrict__ visits,
                  int n_buckets, int *status) {
    extern __shared__ __align__(16) float smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int dim = 2 * K;
    KdNode *nodes_s = reinterpret_cast<KdNode *>(smem);
    const int node_floats = nodes_in_smem ? n_nodes * 4 : 0;
    float *qv = smem + node_floats + warp * dim;
    int *stk_node = reinterpret_cast<int *>(smem + node_floats + KD_WARPS * dim) + warp * kMaxDepth;
    float *stk_bound = reinterpret_cast<float *>(smem + node_floats + KD_WARPS * dim + KD_WARPS * kMaxDepth) +
                       warp * kMaxDepth;
    if (nodes_in_smem) {
        for (int i = threadIdx.x; i < n_nodes; i += blockDim.x) nodes_s[i] = nodes_g[i];
        __syncthreads();
    }
    const KdNode *nodes = nodes_in_smem ? nodes_s : nodes_g;
    for (long long t = (long long)blockIdx.x * KD_WARPS + warp; t < T; t += (long long)gridDim.x * KD_WARPS) {
        // query: conj(Z / ||Z||) embedded as [Re, -Im]
        float n2 = 0.f;
        for (int k = lane; k < K; k += 32) {
            const float2 z = Z[(size_t)t * K + k];
            n2 += z.x * z.x + z.y * z.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
        if (!(n2 > 0.f) || !isfinite(n2)) {
            if (lane == 0) {
                idx_out[t] = -1;
                if (proj_out) proj_out[t] = __int_as_float(0x7fc00000);
                if (visits) {
                    visits[2 * t] = 0;
                    visits[2 * t + 1] = 0;
                }
            }
            continue;
        }
        const float inv = rsqrtf(n2);
        __syncwarp();   // the previous query's reads of qv are done
        for (int k = lane; k < K; k += 32) {
            const float2 z = Z[(size_t)t * K + k];
            qv[k] = z.x * inv;
            qv[K + k] = -z.y * inv;
        }
        __syncwarp();
        float best_d = __int_as_float(0x7f800000);
        int best_id = 0x7fffffff;
        int n_nodes_seen = 0, n_leaves = 0;
        if (lane == 0) {
            stk_node[0] = 0;
            stk_bound[0] = 0.f;
        }
        int sp = 1;
        __syncwarp();
        while (sp > 0) {
            --sp;
            int node = stk_node[sp];
            float bound = stk_bound[sp];
            __syncwarp();
            if (bound > best_d) continue;
            if (!dcheck(node >= 0 && node < n_nodes, status)) continue;
            KdNode nd = nodes[node];
            ++n_nodes_seen;
            while (nd.dim >= 0) {
                if (!dcheck(nd.dim < dim, status)) break;
                const float diff = qv[nd.dim] - nd.split;
                const int near_c = diff < 0.f ? node + 1 : nd.right;
                const int far_c = diff < 0.f ? nd.right : node + 1;
                const float fb = fmaxf(bound, diff * diff);
                if (fb <= best_d && sp < kMaxDepth) {
                    if (lane == 0) {
                        stk_node[sp] = far_c;
                        stk_bound[sp] = fb;
                    }
                    ++sp;
                }
                node = near_c;
                if (!dcheck(node >= 0 && node < n_nodes, status)) break;
                nd = nodes[node];
                ++n_nodes_seen;
            }
            __syncwarp();
            if (nd.dim >= 0) continue;   // only after a failed debug check
            // leaf bucket: lane j scores point j
            ++n_leaves;
            const int bucket = nd.right;
            if (!dcheck(bucket >= 0 && bucket < n_buckets, status)) continue;
            const float *pb = leaf_pts + (size_t)bucket * dim * 32 + lane;
            // four partial sums over interleaved dimensions, eight loads in flight per lane
            float s4[4] = {0.f, 0.f, 0.f, 0.f};
            int d = 0;
            for (; d + 8 <= dim; d += 8) {
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = __ldg(pb + (size_t)(d + u) * 32);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float df = qv[d + u] - v[u];
                    s4[u & 3] = fmaf(df, df, s4[u & 3]);
                }
            }
            for (; d < dim; ++d) {
                const float df = qv[d] - pb[(size_t)d * 32];
                s4[0] = fmaf(df, df, s4[0]);
            }
            float d2 = (s4[0] + s4[1]) + (s4[2] + s4[3]);
            int id = leaf_ids[(size_t)bucket * 32 + lane];
            if (id < 0) {
                d2 = __int_as_float(0x7f800000);
                id = 0x7fffffff;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float od = __shfl_xor_sync(0xffffffffu, d2, o);
                const int oi = __shfl_xor_sync(0xffffffffu, id, o);
                if (od < d2 || (od == d2 && oi < id)) {
                    d2 = od;
                    id = oi;
                }
            }
            if (d2 < best_d || (d2 == best_d && id < best_id)) {
                best_d = d2;
                best_id = id;
            }
        }
        if (lane == 0) {
            idx_out[t] = best_id == 0x7fffffff ? -1 : best_id;
            if (proj_out) proj_out[t] = 1.f - 0.5f * best_d;
            if (visits) {
                visits[2 * t] = n_nodes_seen;
                visits[2 * t + 1] = n_leaves;
            }
        }
    }
}

int launch_kdtree_stats(const sp_basis *b, const void *Z, int T, int32_t *idx, float *proj, int32_t *visits,
                        cudaStream_t s) {
    if (T == 0) return SP_OK;
    const int dim = 2 * b->K;
    const size_t node_bytes = (size_t)b->n_nodes * sizeof(KdNode);
    const int in_smem = node_bytes <= (size_t)kNodeSmem ? 1 : 0;
    const size_t smem = (in_smem ? node_bytes : 0) + (size_t)KD_WARPS * dim * 4 + (size_t)KD_WARPS * kMaxDepth * 8;
    SP_CHECK(smem <= 232448, SP_ENOTIMPL, "k-d tree: shared-memory plan exceeds 227 KB");
    if (smem > 48 * 1024) SP_TRY(ensure_max_smem((const void *)kdtree_kernel));
    const long long need = ((long long)T + KD_WARPS - 1) / KD_WARPS;
    const unsigned grid = (unsigned)std::min<long long>(need, 8LL * num_sms());
    int *status = nullptr;
    SP_TRY(device_status_ptr(&status));
    kdtree_kernel<<<grid, KD_WARPS * 32, smem, s>>>((const float2 *)Z, T, b->K, b->nodes.as<KdNode>(), b->n_nodes,
                                                     in_smem, b->leaf_pts.as<float>(), b->leaf_ids.as<int32_t>(),
                                                     idx, proj, visits, b->n_slots / 32, status);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

int launch_kdtree(const sp_basis *b, const void *Z, int T, int32_t *idx, float *proj, cudaStream_t s) {
    return launch_kdtree_stats(b, Z, T, idx, proj, nullptr, s);
}

}  // namespace sp

using namespace sp;

extern "C" int sp_kdtree_search(const sp_basis *b, const void *z_dev, int T, int32_t *idx_dev, float *proj_dev,
                                int32_t *visits_dev, void *stream) {
    SP_CHECK(b, SP_EINVAL, "sp_kdtree_search: null basis");
    SP_CHECK(T >= 0 && T <= (1 << 28), SP_EINVAL, "sp_kdtree_search: T out of range");
    if (T == 0) return SP_OK;
    SP_CHECK(z_dev && (reinterpret_cast<uintptr_t>(z_dev) & 7) == 0, SP_EINVAL,
             "sp_kdtree_search: z_dev NULL or misaligned");
    SP_CHECK(idx_dev && (reinterpret_cast<uintptr_t>(idx_dev) & 3) == 0, SP_EINVAL,
             "sp_kdtree_search: idx_dev NULL or misaligned");
    SP_CHECK(!proj_dev || (reinterpret_cast<uintptr_t>(proj_dev) & 3) == 0, SP_EINVAL,
             "sp_kdtree_search: proj_dev misaligned");
    SP_CHECK(!visits_dev || (reinterpret_cast<uintptr_t>(visits_dev) & 3) == 0, SP_EINVAL,
             "sp_kdtree_search: visits_dev misaligned");
    return launch_kdtree_stats(b, z_dev, T, idx_dev, proj_dev, visits_dev, (cudaStream_t)stream);
}
