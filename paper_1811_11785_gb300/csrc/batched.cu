// Batched localisation: many independent streams (each its own array, grid, basis and
// frame count) in one CUDA-graph launch.  Algorithm 1's online path runs per stream
// exactly as sp_localize runs it; the plan only schedules the streams' kernels as
// independent branches of one graph so that the GPU runs them concurrently, gives every
// stream its own workspace, and picks the launch shape by measurement.
//
// Shapes and buffers are static per plan (the graph holds the pointers): the caller fills
// the frame buffers it passed at creation and launches the plan with sp_batch_run.
//
// Autotuner: candidate launch shapes are (number of graph branches the streams are spread
// over) x (tiles per CTA of the GEMM1 kernel: 1, 2 or 4, i.e. a CTA cap of tiles / d per
// stream) x (with SP_BATCH_TUNE_KERNELS, the GEMM1 kernel: the TMA-fed one where it applies,
// or the register-fed one -- tried only when some stream could use either; the two sum Z's
// terms in different orders); each candidate graph is built and timed
// (one warm-up, three timed launches with CUDA events) and the fastest is kept.  With a tune
// cache set (sp_set_tune_cache) the chosen shape is stored under the batch's signature
// (device, mode, precision, every stream's M, B, K, classes, T and precision) and a later plan
// with the same signature takes it from the file without measuring.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <map>
#include <memory>
#include <utility>
#include <new>
#include <string>
#include <vector>

#include "common.h"

struct sp_batch {
    int n = 0;
    sp_mode mode = SP_MODE_SVD_EXHAUSTIVE;
    std::vector<const sp_basis *> b;
    std::vector<const void *> frames;
    std::vector<int> T;
    std::vector<sp_prec> prec;          // per stream: the requested precision, or FP32 where the
                                        // tensor-core path does not cover the basis
    std::vector<int32_t *> idx;
    std::vector<float *> score, proj;
    std::vector<std::unique_ptr<sp::DevBuf>> work;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaStream_t origin = nullptr;
    cudaGraphExec_t exec = nullptr;
    int branches = 0, tiles_per_cta = 1, proj_variant = 0;
    float ms = 0.f;                     // measured time of one launch (autotuned plans)
    int from_cache = 0;                 // the shape came from the tune cache
    // Groups: streams that share a basis, a precision and 16-byte-aligned frames (two or more
    // each).  A grouped plan copies a group's frames into one buffer, localises them with one
    // call and copies the results back; `solo` lists the streams in no group.
    struct Group {
        std::vector<int> members;
        int T = 0;
        bool want_score = false, want_proj = false;
        std::unique_ptr<sp::DevBuf> frames, out, work;
    };
    std::vector<Group> groups;
    std::vector<int> solo;
    int grouped = 0;                    // the plan runs the groups (1) or every stream alone (0)
    ~sp_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        for (auto s : side) cudaStreamDestroy(s);
        for (auto e : join) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
        if (origin) cudaStreamDestroy(origin);
    }
};

namespace sp {
namespace {

int enqueue_stream(sp_batch *bt, int i, cudaStream_t s, int tiles_per_cta, int proj_variant) {
    const int tiles = (bt->T[i] + 127) / 128;
    const int cap = std::max(1, (tiles + tiles_per_cta - 1) / tiles_per_cta);
    return localize_ws(bt->b[i], bt->frames[i], bt->T[i], bt->mode, bt->prec[i], bt->idx[i], bt->score[i],
                       bt->proj[i], s, *bt->work[i], cap, proj_variant);
}

size_t group_out_stride(int T) { return ((size_t)T * 4 + 255) / 256 * 256; }

// A group: its streams' frames into the group buffer, one localisation, the results back.
int enqueue_group(sp_batch *bt, sp_batch::Group &g, cudaStream_t s, int tiles_per_cta, int proj_variant) {
    const sp_basis *b = bt->b[g.members[0]];
    const size_t fb = (size_t)b->st->M * b->st->B * 8;
    char *gf = g.frames->as<char>();
    size_t off = 0;
    for (int i : g.members) {
        SP_CUDA(cudaMemcpyAsync(gf + off * fb, bt->frames[i], (size_t)bt->T[i] * fb, cudaMemcpyDeviceToDevice, s));
        off += (size_t)bt->T[i];
    }
    const size_t st = group_out_stride(g.T);
    int32_t *gidx = g.out->as<int32_t>();
    float *gscore = reinterpret_cast<float *>(g.out->as<char>() + st);
    float *gproj = reinterpret_cast<float *>(g.out->as<char>() + 2 * st);
    const int tiles = (g.T + 127) / 128;
    const int cap = std::max(1, (tiles + tiles_per_cta - 1) / tiles_per_cta);
    SP_TRY(localize_ws(b, gf, g.T, bt->mode, bt->prec[g.members[0]], gidx, g.want_score ? gscore : nullptr,
                       g.want_proj ? gproj : nullptr, s, *g.work, cap, proj_variant));
    off = 0;
    for (int i : g.members) {
        const size_t nb = (size_t)bt->T[i] * 4;
        SP_CUDA(cudaMemcpyAsync(bt->idx[i], gidx + off, nb, cudaMemcpyDeviceToDevice, s));
        if (bt->score[i]) SP_CUDA(cudaMemcpyAsync(bt->score[i], gscore + off, nb, cudaMemcpyDeviceToDevice, s));
        if (bt->proj[i]) SP_CUDA(cudaMemcpyAsync(bt->proj[i], gproj + off, nb, cudaMemcpyDeviceToDevice, s));
        off += (size_t)bt->T[i];
    }
    return SP_OK;
}

// The batch's signature: device, mode, precision, and a 64-bit FNV-1a hash of every stream's
// (M, B, K, classes, T, precision, TMA-fed GEMM1 applicable).
int plan_key(const sp_batch *bt, std::string *key) {
    int dev = 0, sms = 0, maj = 0, mnr = 0;
    SP_CUDA(cudaGetDevice(&dev));
    SP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SP_CUDA(cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev));
    SP_CUDA(cudaDeviceGetAttribute(&mnr, cudaDevAttrComputeCapabilityMinor, dev));
    uint64_t h = 1469598103934665603ULL;
    auto mix = [&h](long long v) {
        for (int k = 0; k < 8; ++k) {
            h ^= (uint64_t)((v >> (8 * k)) & 0xff);
            h *= 1099511628211ULL;
        }
    };
    for (int i = 0; i < bt->n; ++i) {
        const sp_steering *st = bt->b[i]->st;
        mix(st->M);
        mix(st->B);
        mix(bt->b[i]->K);
        mix((long long)st->reps.size());
        mix(bt->T[i]);
        mix((int)bt->prec[i]);
        mix(proj_tma_applies(bt->b[i], bt->frames[i]) ? 1 : 0);
    }
    char buf[160];
    std::snprintf(buf, sizeof(buf), "sm%d%d-%dsm/mode%d/prec%d/n%d/%016llx", maj, mnr, sms, (int)bt->mode,
                  bt->n > 0 ? (int)bt->prec[0] : 0, bt->n, (unsigned long long)h);
    *key = buf;
    return SP_OK;
}

// Capture the plan's units into one graph: unit u on branch u % branches.  Units: every
// stream alone, or (grouped) the groups, then the streams in no group.
int build_graph(sp_batch *bt, int branches, int tiles_per_cta, int proj_variant, int grouped, cudaGraphExec_t *out) {
    *out = nullptr;
    while ((int)bt->side.size() < branches) {
        cudaStream_t s;
        cudaEvent_t e;
        SP_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        bt->side.push_back(s);
        SP_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        bt->join.push_back(e);
    }
    cudaGraph_t g = nullptr;
    SP_CUDA(cudaStreamBeginCapture(bt->origin, cudaStreamCaptureModeRelaxed));
    int rc = SP_OK;
    if (cudaEventRecord(bt->fork, bt->origin) != cudaSuccess) rc = fail(SP_ECUDA, "batch: fork record");
    for (int k = 0; k < branches && rc == SP_OK; ++k)
        if (cudaStreamWaitEvent(bt->side[k], bt->fork, 0) != cudaSuccess) rc = fail(SP_ECUDA, "batch: fork wait");
    if (grouped) {
        int u = 0;
        for (size_t gi = 0; gi < bt->groups.size() && rc == SP_OK; ++gi, ++u)
            rc = enqueue_group(bt, bt->groups[gi], bt->side[u % branches], tiles_per_cta, proj_variant);
        for (size_t k = 0; k < bt->solo.size() && rc == SP_OK; ++k, ++u)
            rc = enqueue_stream(bt, bt->solo[k], bt->side[u % branches], tiles_per_cta, proj_variant);
    } else {
        for (int i = 0; i < bt->n && rc == SP_OK; ++i)
            rc = enqueue_stream(bt, i, bt->side[i % branches], tiles_per_cta, proj_variant);
    }
    for (int k = 0; k < branches && rc == SP_OK; ++k) {
        if (cudaEventRecord(bt->join[k], bt->side[k]) != cudaSuccess ||
            cudaStreamWaitEvent(bt->origin, bt->join[k], 0) != cudaSuccess)
            rc = fail(SP_ECUDA, "batch: join");
    }
    const cudaError_t e = cudaStreamEndCapture(bt->origin, &g);
    if (rc != SP_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(SP_ECUDA, std::string("batch: capture: ") + cudaGetErrorString(e));
    const cudaError_t ei = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        *out = nullptr;
        return fail(SP_ECUDA, std::string("batch: instantiate: ") + cudaGetErrorString(ei));
    }
    return SP_OK;
}

int time_graph(cudaGraphExec_t ex, cudaStream_t s, float *ms) {
    cudaEvent_t a, z;
    SP_CUDA(cudaEventCreate(&a));
    SP_CUDA(cudaEventCreate(&z));
    int rc = SP_OK;
    if (cudaGraphLaunch(ex, s) != cudaSuccess || cudaEventRecord(a, s) != cudaSuccess) rc = fail(SP_ECUDA, "batch: launch");
    for (int r = 0; r < 3 && rc == SP_OK; ++r)
        if (cudaGraphLaunch(ex, s) != cudaSuccess) rc = fail(SP_ECUDA, "batch: launch");
    if (rc == SP_OK && (cudaEventRecord(z, s) != cudaSuccess || cudaEventSynchronize(z) != cudaSuccess))
        rc = fail(SP_ECUDA, "batch: timing");
    if (rc == SP_OK) {
        cudaEventElapsedTime(ms, a, z);
        *ms /= 3.f;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    return rc;
}

}  // namespace
}  // namespace sp

using namespace sp;

extern "C" {

int sp_batch_create(int n, const sp_basis *const *bases, const void *const *frames_dev, const int *T, sp_mode mode,
                    sp_prec prec, int32_t *const *idx_dev, float *const *score_dev, float *const *proj_dev, int flags,
                    void *stream, sp_batch **out) {
    SP_CHECK(out, SP_EINVAL, "sp_batch_create: out is NULL");
    *out = nullptr;
    SP_CHECK(n >= 1 && n <= 65536, SP_EINVAL, "sp_batch_create: n must be in [1, 65536]");
    SP_CHECK(bases && frames_dev && T && idx_dev, SP_EINVAL, "sp_batch_create: null array");
    SP_CHECK((flags & ~(SP_BATCH_AUTOTUNE | SP_BATCH_TUNE_KERNELS | SP_BATCH_GROUP)) == 0, SP_EINVAL,
             "sp_batch_create: bad flags");
    SP_CHECK(prec == SP_PREC_FP32 || prec == SP_PREC_FP16 || prec == SP_PREC_BF16, SP_EINVAL,
             "sp_batch_create: bad precision");
    for (int i = 0; i < n; ++i) {
        SP_TRY(check_localize_args(bases[i], frames_dev[i], T[i], idx_dev[i], score_dev ? score_dev[i] : nullptr,
                                   proj_dev ? proj_dev[i] : nullptr));
        SP_CHECK(T[i] >= 1, SP_EINVAL, "sp_batch_create: every stream needs T >= 1");
    }
    std::unique_ptr<sp_batch> bt(new (std::nothrow) sp_batch());
    SP_CHECK(bt, SP_ENOMEM, "sp_batch_create: host allocation failed");
    bt->n = n;
    bt->mode = mode;
    for (int i = 0; i < n; ++i) {
        bt->b.push_back(bases[i]);
        bt->frames.push_back(frames_dev[i]);
        bt->T.push_back(T[i]);
        const bool tc = bases[i]->tc.n1 > 0 && bases[i]->tc_maps;
        bt->prec.push_back(prec != SP_PREC_FP32 && !tc ? SP_PREC_FP32 : prec);
        bt->idx.push_back(idx_dev[i]);
        bt->score.push_back(score_dev ? score_dev[i] : nullptr);
        bt->proj.push_back(proj_dev ? proj_dev[i] : nullptr);
        bt->work.emplace_back(new (std::nothrow) DevBuf());
        SP_CHECK(bt->work.back(), SP_ENOMEM, "sp_batch_create: host allocation failed");
    }
    {   // groups: streams sharing (basis, precision), frames 16-byte aligned, at most 2^28 frames
        std::map<std::pair<const sp_basis *, int>, std::vector<int>> by;
        for (int i = 0; i < n; ++i) {
            if ((reinterpret_cast<uintptr_t>(frames_dev[i]) & 15) != 0) {
                bt->solo.push_back(i);   // an unaligned stream takes its own kernels, as sp_localize does
                continue;
            }
            by[std::make_pair(bases[i], (int)bt->prec[i])].push_back(i);
        }
        for (auto &kv : by) {
            std::vector<int> cur;
            long long Tt = 0;
            auto flush = [&]() -> int {
                if (cur.size() == 1) bt->solo.push_back(cur[0]);
                if (cur.size() >= 2) {
                    sp_batch::Group g;
                    g.members = cur;
                    g.T = (int)Tt;
                    for (int i : cur) {
                        g.want_score = g.want_score || bt->score[i] != nullptr;
                        g.want_proj = g.want_proj || bt->proj[i] != nullptr;
                    }
                    g.frames.reset(new (std::nothrow) DevBuf());
                    g.out.reset(new (std::nothrow) DevBuf());
                    g.work.reset(new (std::nothrow) DevBuf());
                    SP_CHECK(g.frames && g.out && g.work, SP_ENOMEM, "sp_batch_create: host allocation failed");
                    const sp_steering *st = bt->b[cur[0]]->st;
                    SP_TRY(g.frames->reserve((size_t)Tt * st->M * st->B * 8));
                    SP_TRY(g.out->reserve(3 * group_out_stride(g.T)));
                    bt->groups.push_back(std::move(g));
                }
                cur.clear();
                Tt = 0;
                return SP_OK;
            };
            for (int i : kv.second) {
                if (Tt + T[i] > (1LL << 28)) SP_TRY(flush());
                cur.push_back(i);
                Tt += T[i];
            }
            SP_TRY(flush());
        }
        std::sort(bt->solo.begin(), bt->solo.end());
    }
    SP_CUDA(cudaStreamCreateWithFlags(&bt->origin, cudaStreamNonBlocking));
    SP_CUDA(cudaEventCreateWithFlags(&bt->fork, cudaEventDisableTiming));
    // the plan's own stream runs after the work already queued on the caller's stream (which
    // may still be writing the frames, or reading earlier results from the output buffers)
    SP_CUDA(cudaEventRecord(bt->fork, (cudaStream_t)stream));
    SP_CUDA(cudaStreamWaitEvent(bt->origin, bt->fork, 0));
    // one eager pass: sizes every workspace (no allocation happens while capturing) and
    // sets the kernels' attributes
    for (int i = 0; i < n; ++i) SP_TRY(enqueue_stream(bt.get(), i, bt->origin, 1, 0));
    for (auto &g : bt->groups) SP_TRY(enqueue_group(bt.get(), g, bt->origin, 1, 0));
    SP_CUDA(cudaStreamSynchronize(bt->origin));
    const int n_units[2] = {n, (int)(bt->groups.size() + bt->solo.size())};
    auto br_cand = [&](int gv) {
        std::vector<int> c;
        for (int k : {8, 32, 128})
            if (k < n_units[gv]) c.push_back(k);
        c.push_back(n_units[gv]);
        return c;
    };
    const int gv_max = bt->groups.empty() ? 0 : 1;
    if (flags & SP_BATCH_AUTOTUNE) {
        std::string key;
        TunedShape cached{0, 0, 0, 0.f, 0};
        bool found = false;
        if (tune_cache_enabled()) {
            SP_TRY(plan_key(bt.get(), &key));
            key += (flags & SP_BATCH_TUNE_KERNELS) ? "/k" : "";
            if (tune_cache_get(key, &cached, &found) != SP_OK) found = false;   // unreadable file: tune
            if (found && !(cached.grouped >= 0 && cached.grouped <= gv_max && cached.branches >= 1 &&
                           cached.branches <= n_units[cached.grouped] &&
                           (cached.tiles_per_cta == 1 || cached.tiles_per_cta == 2 || cached.tiles_per_cta == 4) &&
                           (cached.proj_variant == 0 || cached.proj_variant == 1)))
                found = false;
        }
        if (found) {
            SP_TRY(build_graph(bt.get(), cached.branches, cached.tiles_per_cta, cached.proj_variant, cached.grouped,
                               &bt->exec));
            bt->grouped = cached.grouped;
            bt->branches = cached.branches;
            bt->tiles_per_cta = cached.tiles_per_cta;
            bt->proj_variant = cached.proj_variant;
            bt->ms = cached.ms;
            bt->from_cache = 1;
        } else {
            bool both = false;   // kernel choice asked for, and some stream could run either GEMM1 kernel
            for (int i = 0; i < n && (flags & SP_BATCH_TUNE_KERNELS); ++i)
                both = both || (bt->prec[i] != SP_PREC_FP32 && proj_tma_applies(bases[i], frames_dev[i]));
            float best = 0.f;
            for (int gv = 0; gv <= gv_max; ++gv)
            for (int pv = 0; pv < (both ? 2 : 1); ++pv)
                for (int br : br_cand(gv))
                    for (int tpc : {1, 2, 4}) {
                        cudaGraphExec_t ex = nullptr;
                        SP_TRY(build_graph(bt.get(), br, tpc, pv, gv, &ex));
                        float ms = 0.f;
                        const int rc = time_graph(ex, bt->origin, &ms);
                        if (rc != SP_OK) {
                            cudaGraphExecDestroy(ex);
                            return rc;
                        }
                        if (!bt->exec || ms < best) {
                            if (bt->exec) cudaGraphExecDestroy(bt->exec);
                            bt->exec = ex;
                            best = ms;
                            bt->branches = br;
                            bt->tiles_per_cta = tpc;
                            bt->proj_variant = pv;
                            bt->grouped = gv;
                        } else {
                            cudaGraphExecDestroy(ex);
                        }
                    }
            bt->ms = best;
            if (!key.empty())
                SP_TRY(tune_cache_put(key, TunedShape{bt->branches, bt->tiles_per_cta, bt->proj_variant, best,
                                                      bt->grouped}));
        }
    } else {
        bt->grouped = (flags & SP_BATCH_GROUP) ? gv_max : 0;   // groups only when asked for
        bt->branches = std::min(n_units[bt->grouped], 32);
        bt->tiles_per_cta = 1;
        SP_TRY(build_graph(bt.get(), bt->branches, 1, 0, bt->grouped, &bt->exec));
    }
    *out = bt.release();
    return SP_OK;
}

int sp_batch_run(sp_batch *bt, void *stream) {
    SP_CHECK(bt && bt->exec, SP_EINVAL, "sp_batch_run: null plan");
    SP_CUDA(cudaGraphLaunch(bt->exec, (cudaStream_t)stream));
    return SP_OK;
}

int sp_batch_info(const sp_batch *bt, int *branches, int *tiles_per_cta, int *proj_variant, float *ms, int *n_fp32,
                  int *from_cache, int *grouped, int *n_groups) {
    SP_CHECK(bt, SP_EINVAL, "sp_batch_info: null plan");
    if (grouped) *grouped = bt->grouped;
    if (n_groups) *n_groups = (int)bt->groups.size();
    if (branches) *branches = bt->branches;
    if (tiles_per_cta) *tiles_per_cta = bt->tiles_per_cta;
    if (proj_variant) *proj_variant = bt->proj_variant;
    if (from_cache) *from_cache = bt->from_cache;
    if (ms) *ms = bt->ms;
    if (n_fp32) {
        int c = 0;
        for (auto p : bt->prec) c += p == SP_PREC_FP32;
        *n_fp32 = c;
    }
    return SP_OK;
}

void sp_batch_destroy(sp_batch *bt) { delete bt; }

int sp_localize_batched(int n, const sp_basis *const *bases, const void *const *frames_dev, const int *T,
                        sp_mode mode, sp_prec prec, int32_t *const *idx_dev, float *const *score_dev,
                        float *const *proj_dev, void *stream) {
    sp_batch *bt = nullptr;
    SP_TRY(sp_batch_create(n, bases, frames_dev, T, mode, prec, idx_dev, score_dev, proj_dev, 0, stream, &bt));
    int rc = sp_batch_run(bt, stream);
    if (rc == SP_OK) {
        const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) rc = fail(SP_ECUDA, std::string("sp_localize_batched: ") + cudaGetErrorString(e));
    }
    sp_batch_destroy(bt);
    return rc;
}

}  // extern "C"
