// C ABI of libsvdphat.so: argument validation, handle lifetime, workspaces and the call
// order of Algorithm 1 (online steps 1-4).  Every step of the path runs in the kernels of
// the other translation units; this file only marshals.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <utility>

#include "common.h"

namespace sp {

static thread_local std::string g_err = "no error";

void set_error(const std::string &msg) { g_err = msg; }
int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

int DevBuf::reserve(size_t n) {
    if (n <= bytes && p) return SP_OK;
    release();
    if (n == 0) return SP_OK;
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        return fail(SP_ENOMEM, std::string("cudaMalloc(") + std::to_string(n) + "): " +
                                   cudaGetErrorString(e));
    }
    bytes = n;
    return SP_OK;
}

static bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

static std::mutex g_dev_mu;

int num_sms() {
    static int cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    std::lock_guard<std::mutex> lock(g_dev_mu);
    if (cache[dev] == 0) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = n > 0 ? n : 1;
    }
    return cache[dev];
}

int ensure_max_smem(const void *kernel) {
    static std::set<std::pair<int, const void *>> done;
    int dev = 0;
    SP_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_dev_mu);
    if (done.count({dev, kernel})) return SP_OK;
    cudaFuncAttributes a;   // the 227 KB per block include the kernel's static shared memory
    SP_CUDA(cudaFuncGetAttributes(&a, kernel));
    SP_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 232448 - (int)a.sharedSizeBytes));
    done.insert({dev, kernel});
    return SP_OK;
}

}  // namespace sp

using namespace sp;

extern "C" {

const char *sp_last_error(void) { return g_err.c_str(); }

int sp_version(void) { return 10000 * 0 + 100 * 1 + 0; }

}  // extern "C"

namespace sp {
// Offline step 1 for far-field directions (Eq. 2) or near-field source positions (Eq. 1).
static int build_steering(const char *fn, const double *mic_xyz, int M, const double *dirs, int Q, double fs,
                          double c, int N, int flags, bool nearfield, sp_steering **out) {
    const std::string name(fn);
    SP_CHECK(out != nullptr, SP_EINVAL, name + ": out is NULL");
    *out = nullptr;
    SP_CHECK(mic_xyz && dirs, SP_EINVAL, name + ": null geometry pointer");
    SP_CHECK(M >= 2 && M <= 64, SP_EINVAL, name + ": M must be in [2, 64]");
    SP_CHECK(Q >= 1 && Q <= (1 << 24), SP_EINVAL, name + ": Q must be in [1, 2^24]");
    SP_CHECK(N >= 4 && N <= 8192 && N % 2 == 0, SP_EINVAL,
             name + ": N must be even and in [4, 8192]");
    SP_CHECK(fs > 0 && c > 0 && std::isfinite(fs) && std::isfinite(c), SP_EINVAL,
             name + ": fs and c must be positive");
    SP_CHECK((flags & ~SP_STEER_MATERIALIZE_W) == 0, SP_EINVAL, name + ": bad flags");
    for (int i = 0; i < 3 * M; ++i)
        SP_CHECK(std::isfinite(mic_xyz[i]), SP_EINVAL, name + ": non-finite mic position");
    for (int q = 0; q < Q; ++q) {
        const double *s = dirs + 3 * q;
        SP_CHECK(std::isfinite(s[0]) && std::isfinite(s[1]) && std::isfinite(s[2]), SP_EINVAL,
                 name + ": non-finite direction");
        SP_CHECK(s[0] != 0 || s[1] != 0 || s[2] != 0, SP_EINVAL,
                 name + (nearfield ? ": source at the coordinate origin" : ": zero direction vector"));
    }
    sp_steering *st = new (std::nothrow) sp_steering();
    SP_CHECK(st != nullptr, SP_ENOMEM, name + ": host allocation failed");
    cudaGetDevice(&st->device);
    st->M = M;
    st->P = M * (M - 1) / 2;
    st->Q = Q;
    st->N = N;
    st->B = N / 2 + 1;
    st->L = st->P * st->B;
    st->fs = fs;
    st->c = c;
    st->mic.assign(mic_xyz, mic_xyz + 3 * M);
    st->dirs.assign(dirs, dirs + 3 * (size_t)Q);
    st->nearfield = nearfield;
    for (int i = 0; i < M; ++i)
        for (int j = i + 1; j < M; ++j) {
            st->pair_i.push_back(i);
            st->pair_j.push_back(j);
        }
    int rc = launch_tau(st, 0);
    if (rc == SP_OK && (flags & SP_STEER_MATERIALIZE_W)) rc = launch_w(st, 0);
    if (rc == SP_OK) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = fail(SP_ECUDA, std::string("build_steering: ") + cudaGetErrorString(e));
    }
    if (rc == SP_OK) {
        st->tau_host.resize((size_t)Q * st->P);
        cudaError_t e = cudaMemcpy(st->tau_host.data(), st->tau.p, st->tau_host.size() * 8,
                                   cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = fail(SP_ECUDA, std::string("build_steering: ") + cudaGetErrorString(e));
    }
    if (rc == SP_OK) rc = build_classes(st);
    if (rc != SP_OK) {
        delete st;
        return rc;
    }
    *out = st;
    return SP_OK;
}
}  // namespace sp

extern "C" {

int sp_build_steering(const double *mic_xyz, int M, const double *dirs, int Q, double fs, double c, int N,
                      int flags, sp_steering **out) {
    return build_steering("sp_build_steering", mic_xyz, M, dirs, Q, fs, c, N, flags, false, out);
}

int sp_build_steering_nearfield(const double *mic_xyz, int M, const double *src_xyz, int Q, double fs, double c,
                                int N, int flags, sp_steering **out) {
    return build_steering("sp_build_steering_nearfield", mic_xyz, M, src_xyz, Q, fs, c, N, flags, true, out);
}

int sp_steering_nearfield(const sp_steering *st, int *nearfield) {
    SP_CHECK(st && nearfield, SP_EINVAL, "sp_steering_nearfield: null pointer");
    *nearfield = st->nearfield ? 1 : 0;
    return SP_OK;
}

int sp_steering_dims(const sp_steering *st, int *M, int *P, int *Q, int *N, int *B) {
    SP_CHECK(st, SP_EINVAL, "sp_steering_dims: null handle");
    if (M) *M = st->M;
    if (P) *P = st->P;
    if (Q) *Q = st->Q;
    if (N) *N = st->N;
    if (B) *B = st->B;
    return SP_OK;
}

int sp_steering_classes(const sp_steering *st, int *n_classes, int32_t *rep_of_host) {
    SP_CHECK(st, SP_EINVAL, "sp_steering_classes: null handle");
    if (n_classes) *n_classes = (int)st->reps.size();
    if (rep_of_host) std::memcpy(rep_of_host, st->rep_of.data(), st->rep_of.size() * sizeof(int32_t));
    return SP_OK;
}

int sp_steering_tau(const sp_steering *st, double *tau_host) {
    SP_CHECK(st && tau_host, SP_EINVAL, "sp_steering_tau: null pointer");
    std::memcpy(tau_host, st->tau_host.data(), st->tau_host.size() * sizeof(double));
    return SP_OK;
}

int sp_steering_w(const sp_steering *st, void *w_dev, void *stream) {
    SP_CHECK(st && w_dev, SP_EINVAL, "sp_steering_w: null pointer");
    SP_CHECK(st->has_w, SP_EINVAL, "sp_steering_w: W was not materialised (SP_STEER_MATERIALIZE_W)");
    SP_CUDA(cudaMemcpyAsync(w_dev, st->W.p, (size_t)st->Q * st->L * 8, cudaMemcpyDeviceToDevice,
                            (cudaStream_t)stream));
    return SP_OK;
}

void sp_steering_destroy(sp_steering *st) { delete st; }

int sp_svd_reduce(const sp_steering *st, double delta, int flags, sp_basis **out, int *K_out) {
    SP_CHECK(out, SP_EINVAL, "sp_svd_reduce: out is NULL");
    *out = nullptr;
    SP_CHECK(st, SP_EINVAL, "sp_svd_reduce: null steering handle");
    SP_CHECK(delta > 0 && delta < 1, SP_EINVAL, "sp_svd_reduce: delta must be in (0, 1)");
    SP_CHECK(flags == 0, SP_EINVAL, "sp_svd_reduce: flags must be 0");
    sp_basis *b = new (std::nothrow) sp_basis();
    SP_CHECK(b != nullptr, SP_ENOMEM, "sp_svd_reduce: host allocation failed");
    b->st = st;
    b->delta = delta;
    int rc = reduce_basis(st, delta, b);
    if (rc == SP_OK) rc = build_kdtree(b);
    if (rc == SP_OK) rc = tc_prepare(b);
    if (rc == SP_OK) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = fail(SP_ECUDA, std::string("svd_reduce: ") + cudaGetErrorString(e));
    }
    if (rc != SP_OK) {
        delete b;
        return rc;
    }
    if (K_out) *K_out = b->K;
    *out = b;
    return SP_OK;
}

int sp_basis_info(const sp_basis *b, int *K, int *n_sigma, double *sigma2_host, int cap) {
    SP_CHECK(b, SP_EINVAL, "sp_basis_info: null handle");
    if (K) *K = b->K;
    if (n_sigma) *n_sigma = (int)b->sigma2.size();
    if (sigma2_host && cap > 0) {
        int n = std::min<int>(cap, (int)b->sigma2.size());
        std::memcpy(sigma2_host, b->sigma2.data(), n * sizeof(double));
    }
    return SP_OK;
}

int sp_basis_v(const sp_basis *b, double *v_host) {
    SP_CHECK(b && v_host, SP_EINVAL, "sp_basis_v: null pointer");
    std::memcpy(v_host, b->V.data(), b->V.size() * sizeof(double));
    return SP_OK;
}

int sp_basis_d(const sp_basis *b, double *d_host) {
    SP_CHECK(b && d_host, SP_EINVAL, "sp_basis_d: null pointer");
    std::memcpy(d_host, b->D.data(), b->D.size() * sizeof(double));
    return SP_OK;
}

int sp_basis_kdtree_info(const sp_basis *b, int *n_nodes, int *leaf_size, int *depth) {
    SP_CHECK(b, SP_EINVAL, "sp_basis_kdtree_info: null handle");
    if (n_nodes) *n_nodes = b->n_nodes;
    if (leaf_size) *leaf_size = b->leaf_size;
    if (depth) *depth = b->depth;
    return SP_OK;
}

void sp_basis_destroy(sp_basis *b) { delete b; }

int sp_phat(const void *frames_dev, int T, int M, int B, void *x_dev, void *stream) {
    SP_CHECK(T >= 0, SP_EINVAL, "sp_phat: T < 0");
    SP_CHECK(M >= 2 && M <= 64 && B >= 1, SP_EINVAL, "sp_phat: bad M or B");
    if (T == 0) return SP_OK;
    SP_CHECK(frames_dev && x_dev, SP_EINVAL, "sp_phat: null pointer");
    SP_CHECK(aligned(frames_dev, 8) && aligned(x_dev, 8), SP_EINVAL, "sp_phat: pointers must be 8-byte aligned");
    return launch_phat(frames_dev, T, M, B, x_dev, (cudaStream_t)stream);
}

static int check_frames(const sp_steering *st, const void *frames, int T) {
    SP_CHECK(T >= 0, SP_EINVAL, "T < 0");
    SP_CHECK(T <= (1 << 28), SP_EINVAL, "T too large");
    SP_CHECK(T == 0 || frames, SP_EINVAL, "frames pointer is NULL");
    SP_CHECK(aligned(frames, 8), SP_EINVAL, "frames must be 8-byte aligned");
    SP_CHECK(st->M <= 16, SP_ENOTIMPL, "localisation kernels support M <= 16 microphones");
    return SP_OK;
}

int sp_project(const sp_basis *b, const void *frames_dev, int T, sp_prec prec, void *z_dev,
               void *stream) {
    SP_CHECK(b, SP_EINVAL, "sp_project: null basis");
    SP_TRY(check_frames(b->st, frames_dev, T));
    if (T == 0) return SP_OK;
    SP_CHECK(z_dev && aligned(z_dev, 8), SP_EINVAL, "sp_project: z_dev NULL or misaligned");
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == SP_PREC_FP32) {
        const sp_steering *st = b->st;
        SP_TRY(b->work.reserve((size_t)T * st->L * 8));
        SP_TRY(launch_phat(frames_dev, T, st->M, st->B, b->work.p, s));
        return launch_project_f32(b, b->work.p, T, z_dev, s);
    }
    SP_CHECK(prec == SP_PREC_FP16 || prec == SP_PREC_BF16, SP_EINVAL, "sp_project: bad precision");
    return launch_svd_proj(b, frames_dev, T, (int)prec, z_dev, nullptr, s);
}

static int srp_path(const sp_steering *st, const void *frames, int T, int32_t *idx, float *best,
                    DevBuf &work, cudaStream_t s) {
    SP_CHECK(st->has_w, SP_ENOTIMPL, "SRP needs a materialised W (SP_STEER_MATERIALIZE_W)");
    const size_t xbytes = ((size_t)T * st->L * 8 + 255) / 256 * 256;
    SP_TRY(work.reserve(xbytes + (size_t)T * 8));
    uint64_t *keys = reinterpret_cast<uint64_t *>(work.as<char>() + xbytes);
    SP_TRY(launch_phat(frames, T, st->M, st->B, work.p, s));
    return launch_srp_argmax(st->W.p, st->Q, st->L, work.p, T, keys, idx, best, s);
}

}  // extern "C"

namespace sp {

// The online path of one batch of frames with an explicit workspace (sp_localize uses the
// basis's own; a batch plan gives every stream its own so that streams run concurrently).
// max_ctas > 0 caps the CTAs of the tensor-core GEMM1 kernel (tiles per CTA = tiles / cap).
int localize_ws(const sp_basis *b, const void *frames_dev, int T, sp_mode mode, sp_prec prec, int32_t *idx_dev,
                float *score_dev, float *proj_score_dev, cudaStream_t s, DevBuf &work, int max_ctas,
                int proj_variant) {
    const sp_steering *st = b->st;
    switch (mode) {
        case SP_MODE_SRP: {
            SP_CHECK(prec == SP_PREC_FP32, SP_ENOTIMPL, "SRP runs in FP32 only");
            SP_TRY(srp_path(st, frames_dev, T, idx_dev, proj_score_dev, work, s));
            break;
        }
        case SP_MODE_SVD_EXHAUSTIVE: {
            if (prec == SP_PREC_FP32) {
                const size_t xbytes = ((size_t)T * st->L * 8 + 255) / 256 * 256;
                const size_t zbytes = ((size_t)T * b->K * 8 + 255) / 256 * 256;
                SP_TRY(work.reserve(xbytes + zbytes + (size_t)T * 8));
                char *w = work.as<char>();
                SP_TRY(launch_phat(frames_dev, T, st->M, st->B, w, s));
                SP_TRY(launch_project_f32(b, w, T, w + xbytes, s));
                SP_TRY(launch_svd_scan_f32(b, w + xbytes, T, reinterpret_cast<uint64_t *>(w + xbytes + zbytes),
                                           idx_dev, proj_score_dev, s));
            } else {
                SP_CHECK(prec == SP_PREC_FP16 || prec == SP_PREC_BF16, SP_EINVAL, "bad precision");
                const size_t zbytes = ((size_t)T * b->K * 8 + 255) / 256 * 256;
                const size_t nbytes = ((size_t)T * 4 + 255) / 256 * 256;
                SP_TRY(work.reserve(zbytes + nbytes + scan_workspace_bytes(T)));
                float *zn2 = reinterpret_cast<float *>(work.as<char>() + zbytes);
                SP_TRY(launch_svd_proj(b, frames_dev, T, (int)prec, work.p, zn2, s, max_ctas, proj_variant));
                SP_TRY(launch_svd_scan(b, work.p, zn2, T, (int)prec, idx_dev, proj_score_dev, s,
                                       work.as<char>() + zbytes + nbytes));
            }
            break;
        }
        case SP_MODE_SVD_KDTREE: {
            const size_t zbytes = ((size_t)T * b->K * 8 + 255) / 256 * 256;
            if (prec == SP_PREC_FP32) {
                const size_t xbytes = ((size_t)T * st->L * 8 + 255) / 256 * 256;
                SP_TRY(work.reserve(xbytes + zbytes));
                char *w = work.as<char>();
                SP_TRY(launch_phat(frames_dev, T, st->M, st->B, w, s));
                SP_TRY(launch_project_f32(b, w, T, w + xbytes, s));
                SP_TRY(launch_kdtree(b, w + xbytes, T, idx_dev, proj_score_dev, s));
            } else {
                SP_CHECK(prec == SP_PREC_FP16 || prec == SP_PREC_BF16, SP_EINVAL, "bad precision");
                SP_TRY(work.reserve(zbytes));
                SP_TRY(launch_svd_proj(b, frames_dev, T, (int)prec, work.p, nullptr, s, max_ctas, proj_variant));
                SP_TRY(launch_kdtree(b, work.p, T, idx_dev, proj_score_dev, s));
            }
            break;
        }
        case SP_MODE_SVD_LEARNED:
            return fail(SP_EINVAL, "SP_MODE_SVD_LEARNED needs a proposal: call sp_localize_learned");
        default:
            return fail(SP_EINVAL, "sp_localize: bad mode");
    }
    if (score_dev) SP_TRY(launch_score_row(st, frames_dev, T, idx_dev, score_dev, s));
    return SP_OK;
}

int check_localize_args(const sp_basis *b, const void *frames_dev, int T, const int32_t *idx_dev,
                        const float *score_dev, const float *proj_score_dev) {
    SP_CHECK(b, SP_EINVAL, "sp_localize: null basis");
    SP_TRY(check_frames(b->st, frames_dev, T));
    if (T == 0) return SP_OK;
    SP_CHECK(idx_dev && aligned(idx_dev, 4), SP_EINVAL, "sp_localize: idx_dev NULL or misaligned");
    SP_CHECK(!score_dev || aligned(score_dev, 4), SP_EINVAL, "sp_localize: score_dev misaligned");
    SP_CHECK(!proj_score_dev || aligned(proj_score_dev, 4), SP_EINVAL,
             "sp_localize: proj_score_dev misaligned");
    return SP_OK;
}

}  // namespace sp

extern "C" {

int sp_localize(const sp_basis *b, const void *frames_dev, int T, sp_mode mode, sp_prec prec,
                int32_t *idx_dev, float *score_dev, float *proj_score_dev, void *stream) {
    SP_TRY(check_localize_args(b, frames_dev, T, idx_dev, score_dev, proj_score_dev));
    if (T == 0) return SP_OK;
    return localize_ws(b, frames_dev, T, mode, prec, idx_dev, score_dev, proj_score_dev, (cudaStream_t)stream,
                       b->work, 0);
}

int sp_localize_srp(const sp_steering *st, const void *frames_dev, int T, int32_t *idx_dev,
                    float *score_dev, void *stream) {
    SP_CHECK(st, SP_EINVAL, "sp_localize_srp: null steering");
    SP_TRY(check_frames(st, frames_dev, T));
    if (T == 0) return SP_OK;
    SP_CHECK(idx_dev && aligned(idx_dev, 4), SP_EINVAL, "sp_localize_srp: idx_dev NULL or misaligned");
    SP_CHECK(!score_dev || aligned(score_dev, 4), SP_EINVAL, "sp_localize_srp: score_dev misaligned");
    return srp_path(st, frames_dev, T, idx_dev, score_dev, st->work, (cudaStream_t)stream);
}

int sp_localize_host(const sp_basis *b, const void *frames_host, int T, sp_mode mode,
                     sp_prec prec, int32_t *idx_host, float *score_host, float *proj_score_host,
                     int chunk_frames, void *stream) {
    SP_CHECK(b, SP_EINVAL, "sp_localize_host: null basis");
    const sp_steering *st = b->st;
    SP_CHECK(T >= 0, SP_EINVAL, "sp_localize_host: T < 0");
    if (T == 0) return SP_OK;
    SP_CHECK(frames_host && idx_host, SP_EINVAL, "sp_localize_host: null pointer");
    if (chunk_frames <= 0) chunk_frames = 16384;
    chunk_frames = std::min(chunk_frames, T);
    const size_t fbytes = (size_t)st->M * st->B * 8;        // one frame of STFT
    const size_t in_bytes = ((size_t)chunk_frames * fbytes + 255) / 256 * 256;
    const size_t out_bytes = (size_t)chunk_frames * 12;     // idx, score, proj
    for (int i = 0; i < 2; ++i) SP_TRY(b->stage[i].reserve(in_bytes + out_bytes));
    cudaStream_t s0 = (cudaStream_t)stream;
    if (!b->copy_stream) {
        SP_CUDA(cudaStreamCreateWithFlags(&b->copy_stream, cudaStreamNonBlocking));
        for (int i = 0; i < 2; ++i) {
            SP_CUDA(cudaEventCreateWithFlags(&b->ev_loaded[i], cudaEventDisableTiming));
            SP_CUDA(cudaEventCreateWithFlags(&b->ev_free[i], cudaEventDisableTiming));
        }
    }
    // Two staging buffers.  Chunk c's frames are copied on the copy stream (after the
    // kernels of chunk c-2, which used the same buffer, are done) while the compute stream
    // localises chunk c-1; results come back on the compute stream.
    const int nchunks = (T + chunk_frames - 1) / chunk_frames;
    SP_CUDA(cudaEventRecord(b->ev_free[0], s0));
    SP_CUDA(cudaEventRecord(b->ev_free[1], s0));
    for (int c = 0; c < nchunks; ++c) {
        const int t0 = c * chunk_frames;
        const int n = std::min(chunk_frames, T - t0);
        const int u = c & 1;
        DevBuf &sb = b->stage[u];
        char *dframes = sb.as<char>();
        int32_t *didx = reinterpret_cast<int32_t *>(dframes + in_bytes);
        float *dscore = reinterpret_cast<float *>(didx + chunk_frames);
        float *dproj = dscore + chunk_frames;
        SP_CUDA(cudaStreamWaitEvent(b->copy_stream, b->ev_free[u], 0));
        SP_CUDA(cudaMemcpyAsync(dframes, (const char *)frames_host + (size_t)t0 * fbytes,
                                (size_t)n * fbytes, cudaMemcpyHostToDevice, b->copy_stream));
        SP_CUDA(cudaEventRecord(b->ev_loaded[u], b->copy_stream));
        SP_CUDA(cudaStreamWaitEvent(s0, b->ev_loaded[u], 0));
        SP_TRY(sp_localize(b, dframes, n, mode, prec, didx, score_host ? dscore : nullptr,
                           proj_score_host ? dproj : nullptr, s0));
        SP_CUDA(cudaMemcpyAsync(idx_host + t0, didx, (size_t)n * 4, cudaMemcpyDeviceToHost, s0));
        if (score_host)
            SP_CUDA(cudaMemcpyAsync(score_host + t0, dscore, (size_t)n * 4, cudaMemcpyDeviceToHost, s0));
        if (proj_score_host)
            SP_CUDA(cudaMemcpyAsync(proj_score_host + t0, dproj, (size_t)n * 4, cudaMemcpyDeviceToHost, s0));
        SP_CUDA(cudaEventRecord(b->ev_free[u], s0));
    }
    SP_CUDA(cudaStreamSynchronize(s0));
    return SP_OK;
}

int sp_localize_samples(const sp_basis *b, const float *samples_dev, long long n_samples, long long ld, int hop,
                        const uint8_t *mask_dev, int T, sp_mode mode, sp_prec prec, int32_t *idx_dev,
                        float *score_dev, float *proj_score_dev, void *stream) {
    SP_CHECK(b, SP_EINVAL, "sp_localize_samples: null basis");
    const sp_steering *st = b->st;
    SP_TRY(check_stft_args(samples_dev, st->M, n_samples, ld, st->N, hop));
    SP_CHECK(T >= 0 && T <= stft_frames(n_samples, st->N, hop), SP_EINVAL,
             "sp_localize_samples: T exceeds the whole frames in the samples");
    if (T == 0) return SP_OK;
    SP_CHECK(idx_dev && aligned(idx_dev, 4), SP_EINVAL, "sp_localize_samples: idx_dev NULL or misaligned");
    SP_CHECK(!score_dev || aligned(score_dev, 4), SP_EINVAL, "sp_localize_samples: score_dev misaligned");
    SP_CHECK(!proj_score_dev || aligned(proj_score_dev, 4), SP_EINVAL,
             "sp_localize_samples: proj_score_dev misaligned");
    SP_TRY(b->fe_frames.reserve((size_t)T * st->M * st->B * 8));
    cudaStream_t s = (cudaStream_t)stream;
    SP_TRY(launch_stft(samples_dev, ld, st->M, st->N, hop, T, mask_dev, b->fe_frames.p, s));
    return sp_localize(b, b->fe_frames.p, T, mode, prec, idx_dev, score_dev, proj_score_dev, stream);
}

int sp_check_status(void *stream) {
    int status = 0;
    SP_TRY(read_and_clear_device_status((cudaStream_t)stream, &status));
    if (status & 0x100)
        return fail(SP_EBOUNDS, "a device bounds check of the debug build failed (status " + std::to_string(status) + ")");
    if (status != 0)
        return fail(SP_ETIMEOUT, "a bounded device wait gave up (status " + std::to_string(status) + ")");
    return SP_OK;
}

}  // extern "C"
