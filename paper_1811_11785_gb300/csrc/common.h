// Internal declarations shared by the translation units of libsvdphat.so.
// Host-side only (no device code); kernels live in the .cu files and are reached
// through the launch_* functions declared here.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/svdphat.h"

namespace sp {

// ---------------------------------------------------------------- error plumbing
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);

#define SP_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return ::sp::fail(SP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define SP_CHECK(cond, code, msg)                                                       \
    do {                                                                                \
        if (!(cond)) return ::sp::fail((code), (msg));                                  \
    } while (0)

#define SP_TRY(call)                                                                    \
    do {                                                                                \
        int r_ = (call);                                                                \
        if (r_ != SP_OK) return r_;                                                     \
    } while (0)

// ---------------------------------------------------------------- device buffers
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    // grow-only; contents are not preserved
    int reserve(size_t n);
    template <class T> T *as() const { return reinterpret_cast<T *>(p); }
};

// ---------------------------------------------------------------- device status word
// Set by kernels whose bounded waits gave up (see sp_check_status).
int read_and_clear_device_status(cudaStream_t s, int *status);
long long wait_budget();
int device_status_ptr(int **out);   // the status word's device address (current device)

// ---------------------------------------------------------------- tiling of the
// tensor-core projection (K-dimension layout of GEMM1, chosen for the GPU; the paper's
// Eq. 7 column order p*B + k is a different permutation of the same contraction index).
//   chunk c covers bins 4c .. 4c+3; inside a chunk, pair p and bin b sit at element
//   p*8 + 2b (+0 real, +1 imaginary); a chunk spans kAtomsPerChunk 64-element atoms.
constexpr int kChunkBins = 4;
struct TcLayout {
    int P = 0, Pp = 0;            // pairs and pairs rounded up to even
    int steps_per_chunk = 0;      // K16 MMA steps per chunk = Pp / 2
    int atoms_per_chunk = 0;      // 64-element swizzle atoms per chunk
    int n_chunks = 0;             // ceil(B / 4)
    int row_elems = 0;            // n_chunks * atoms_per_chunk * 64
    int n1 = 0;                   // GEMM1 N = 2K rounded up to a multiple of 16
    int k2 = 0;                   // GEMM2 K = 2K rounded up to 16
    int k2_atoms = 0;             // 64-element atoms of the GEMM2 K dimension
    int n2 = 128;                 // Q tile of GEMM2
    int v_box = 0;                // rows per TMA box of a V atom (n1, or n1 / 2 when n1 > 256)
};
TcLayout make_tc_layout(int P, int B, int K);

// ---------------------------------------------------------------- k-d tree
struct KdNode {               // 16 bytes
    int32_t dim;              // split dimension, or -1 for a leaf
    float split;              // split value (points with x[dim] < split go left)
    int32_t right;            // index of the right child (left child is this + 1); leaf: first slot
    int32_t count;            // leaf: number of points in the bucket (0 for internal nodes)
};

// ---------------------------------------------------------------- handles
}  // namespace sp

struct sp_basis;
namespace sp {
void tc_release(sp_basis *b);  // frees the tensor maps of the tensor-core path
}

struct sp_steering {
    int device = 0;
    int M = 0, P = 0, Q = 0, N = 0, B = 0, L = 0;
    double fs = 0, c = 0;
    std::vector<double> mic, dirs;      // host copies (M x 3, Q x 3)
    bool nearfield = false;             // dirs are source positions and tau follows Eq. 1
    std::vector<int> pair_i, pair_j;    // Eq. 7 pair order
    std::vector<double> tau_host;       // Q x P
    // Directions whose TDOA vectors agree within 1e-9 samples have identical rows of W
    // (and of D), hence identical scores for every observation; each such class is
    // scanned once, at its lowest index.  reps: the class representatives, ascending.
    std::vector<int> rep_of;            // Q: representative (lowest index) of q's class
    std::vector<int> reps;              // n_classes representatives
    sp::DevBuf d_reps;                  // int32 [n_classes]
    sp::DevBuf tau;                     // Q x P double
    sp::DevBuf d_mic;                   // M x 3 double
    sp::DevBuf d_dirs;                  // Q x 3 double (unit directions, for step 4)
    sp::DevBuf step4_tab;               // Q x M float4: d_m/N (hi, lo), 64-bin step phasor
    sp::DevBuf W;                       // Q x L complex64 (optional)
    bool has_w = false;
    mutable sp::DevBuf work;            // workspace for SRP calls on this handle
};

struct sp_basis {
    const sp_steering *st = nullptr;
    int K = 0;
    double delta = 0;
    std::vector<double> sigma2;         // Ritz values, descending
    std::vector<double> V, D;           // host FP64 complex, L x K and Q x K (interleaved)
    // device copies
    sp::DevBuf Vc32;                    // V^T as complex64 [K][L], column l = p*B + k (Eq. 7 order)
    sp::DevBuf Dc32;                    // D as complex64 [Q][K]
    sp::DevBuf Dc32r;                   // D rows of the class representatives [n_classes][K]
    sp::TcLayout tc;
    sp::DevBuf Vtc[2];                  // GEMM1 B operand, fp16 [0] / bf16 [1]: [n1][row_elems]
    sp::DevBuf Vbm[2];                  // the same with bin-major chunks (pair p, bin b of a chunk at
                                        // element 48 b + 2 p) for the TMA-fed GEMM1 (M = 7); else empty
    sp::DevBuf Dtc[2];                  // GEMM2 B operand, fp16 / bf16: [Q][k2_atoms*64]
    float v_scale = 1.f;                // Vtc holds V * v_scale
    void *tc_maps = nullptr;            // TMA descriptors of Vtc / Dtc (owned)
    // k-d tree over the rows [Re D^_q, Im D^_q]
    std::vector<sp::KdNode> nodes_host;
    sp::DevBuf nodes;                   // KdNode[n_nodes]
    sp::DevBuf leaf_pts;                // float [n_slots/32][2K][32] bucket-major, dimension-major
    sp::DevBuf leaf_ids;                // int32 [n_slots]
    int n_nodes = 0, leaf_size = 32, depth = 0, n_slots = 0;
    mutable sp::DevBuf work;            // workspace for localize calls
    mutable sp::DevBuf stage[2];        // host-path staging
    mutable sp::DevBuf fe_frames;       // STFT frames of sp_localize_samples
    mutable cudaStream_t copy_stream = nullptr;      // host-path copies
    mutable cudaEvent_t ev_loaded[2] = {nullptr, nullptr};
    mutable cudaEvent_t ev_free[2] = {nullptr, nullptr};
    sp_steering *owned_st = nullptr;   // set when the basis was loaded from a file
    ~sp_basis() {
        sp::tc_release(this);
        for (int i = 0; i < 2; ++i) {
            if (ev_loaded[i]) cudaEventDestroy(ev_loaded[i]);
            if (ev_free[i]) cudaEventDestroy(ev_free[i]);
        }
        if (copy_stream) cudaStreamDestroy(copy_stream);
        delete owned_st;
    }
};

namespace sp {
// launchers implemented in the .cu files ------------------------------------------
int launch_tau(const sp_steering *st, cudaStream_t s);
int launch_w(const sp_steering *st, cudaStream_t s);
int launch_phat(const void *frames, int T, int M, int B, void *x, cudaStream_t s);
// Y = Re{A_q . X_t} over contraction length Lc (A: [Qa][Lc] complex64, X: [T][Lc] complex64),
// argmax over q per frame -> idx / best (keys scratch: T x uint64).
int launch_srp_argmax(const void *A, int Qa, int Lc, const void *X, int T, uint64_t *keys,
                      int32_t *idx, float *best, cudaStream_t s);
int launch_project_f32(const sp_basis *b, const void *X, int T, void *Z, cudaStream_t s);
int launch_svd_scan_f32_list(const sp_basis *b, const void *Z, int T_cap, const int *count, const int32_t *list,
                             uint64_t *keys, int32_t *idx, float *best, cudaStream_t s);
int launch_svd_scan_f32(const sp_basis *b, const void *Z, int T, uint64_t *keys, int32_t *idx,
                        float *best, cudaStream_t s);
int launch_score_row(const sp_steering *st, const void *frames, int T, const int32_t *idx,
                     float *score, cudaStream_t s);
int launch_step4_bulk(const sp_steering *st, const void *frames, int T, const int32_t *idx, float *score,
                      cudaStream_t s);   // SP_ENOTIMPL where its plan does not apply
// tensor-core path: Z = V^H X (PHAT fused) into z_out [T][K] complex64, then the Re{D Z} scan
// (zn2_out [T] receives ||Z||^2 per frame, may be null; the scan needs it)
// proj_variant: 0 = the TMA-fed kernel where its plan applies (7 microphones), else the
// register-fed one; 1 = always the register-fed kernel
int launch_svd_proj(const sp_basis *b, const void *frames, int T, int prec, void *z_out, float *zn2_out,
                    cudaStream_t s, int max_ctas = 0, int proj_variant = 0);
// ws: scan_workspace_bytes(T) bytes, 256-byte aligned (list of the frames whose candidate
// window overflows, their keys and a count).  With rows/n_rows (device) only the frames
// rows[0 .. *n_rows) of Z's T frames are scanned (and only their idx/proj written).
size_t scan_workspace_bytes(int T);
int launch_svd_scan(const sp_basis *b, const void *Z, const float *zn2, int T, int prec, int32_t *idx,
                    float *proj, cudaStream_t s, void *ws, const int32_t *rows = nullptr,
                    const int *n_rows = nullptr);
int launch_kdtree(const sp_basis *b, const void *Z, int T, int32_t *idx, float *proj,
                  cudaStream_t s);
int tc_prepare(sp_basis *b);
// TMA descriptor of the bin-major GEMM1 B operand (Vbm) of a basis, fp16 (bf16 = 0) or bf16;
// null where the basis has none
const CUtensorMap *tc_vmap_binmajor(const sp_basis *b, int bf16);
// GEMM1 with the STFT fed by TMA (7 microphones, odd B, 16-byte-aligned frames); SP_ENOTIMPL
// where its plan does not apply, and the caller then runs svd_proj_kernel / svd_proj_tm_kernel
int launch_svd_proj_tma(const sp_basis *b, const void *frames, int T, int prec, void *z_out, float *zn2_out,
                        cudaStream_t s, int max_ctas);
// Load the kernels a localisation of this basis / array would launch on the current device
// and set their shared-memory limits (what their first launches would otherwise do).
int prepare_tc(const sp_basis *b, int prec);
int prepare_simt(const sp_steering *st);
int prepare_step4(const sp_steering *st);
// 2-D tensor map of a row-major [rows][inner] fp16 (bf16 = 0) / bf16 (bf16 = 1) array,
// 128-byte swizzle, box {box_inner, box_rows}
int encode_tmap_2d(CUtensorMap *map, void *base, int bf16, uint64_t inner, uint64_t rows, uint32_t box_inner,
                   uint32_t box_rows);
// Multiprocessor count of the current device (looked up once per device).
// 2-D tensor map of a float32 array with rows row_stride_bytes apart (a multiple of 16),
// no swizzle, zero fill outside [inner] x [rows], box {box_inner, box_rows}
int encode_tmap_f32_2d(CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows, uint64_t row_stride_bytes,
                       uint32_t box_inner, uint32_t box_rows);
int num_sms();
// Raise a kernel's shared-memory limit (static + dynamic) to 227 KB on the current device.  The
// attribute belongs to the device, so it is set once per (device, kernel) pair; a process
// that drives several GPUs sets it on each.  Thread-safe.
int ensure_max_smem(const void *kernel);
int reduce_basis(const sp_steering *st, double delta, sp_basis *b);
int install_basis(sp_basis *b);   // device copies of b->V, b->D (host FP64, filled)
int build_kdtree(sp_basis *b);
int localize_ws(const sp_basis *b, const void *frames_dev, int T, sp_mode mode, sp_prec prec, int32_t *idx_dev,
                float *score_dev, float *proj_score_dev, cudaStream_t s, DevBuf &work, int max_ctas,
                int proj_variant = 0);
// whether the TMA-fed GEMM1 applies to this basis and frame buffer
bool proj_tma_applies(const sp_basis *b, const void *frames);
// autotune cache of batch plans (tunecache.cu): the file set by sp_set_tune_cache
struct TunedShape {
    int branches, tiles_per_cta, proj_variant;
    float ms;
    int grouped;   // 1: the plan localises groups of streams that share a basis
};
bool tune_cache_enabled();
int tune_cache_get(const std::string &key, TunedShape *out, bool *found);
int tune_cache_put(const std::string &key, const TunedShape &v);
int check_localize_args(const sp_basis *b, const void *frames_dev, int T, const int32_t *idx_dev,
                        const float *score_dev, const float *proj_score_dev);
int build_classes(sp_steering *st);   // rep_of / reps from the TDOA table (host)
// STFT front end (Section 2): number of whole frames, argument checks, launch
int stft_frames(long long n_samples, int N, int hop);
int check_stft_args(const float *x, int M, long long n_samples, long long ld, int N, int hop);
int launch_stft(const float *x, long long ld, int M, int N, int hop, int T, const uint8_t *mask, void *frames,
                cudaStream_t s);
}  // namespace sp
