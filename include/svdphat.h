/*
 * svdphat.h -- C ABI of the GB300 (sm_103a) SVD-PHAT hot path, libsvdphat.so.
 *
 * Method: F. Grondin and J. Glass, "SVD-PHAT: A Fast Sound Source Localization
 * Method" (arXiv 1811.11785).  Section 2 defines SRP-PHAT (Eq. 1-9), Section 3 the
 * SVD-PHAT reduction and search (Eq. 10-15) and Algorithm 1 the offline/online split.
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  - Return value: SP_OK (0) or a negative SP_E* code; sp_last_error() then holds a
 *    one-line message (thread-local).  No C++ exception crosses this boundary.
 *  - Pointers documented as "device" are CUDA device pointers on the current device;
 *    "host" pointers are ordinary (ideally pinned) host memory.  The caller owns every
 *    buffer it passes; the library owns only its opaque handles, which it frees in the
 *    matching *_destroy call.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default stream).  Work
 *    is enqueued asynchronously on it unless stated otherwise; device-side failures
 *    (a bounded wait that gave up) are recorded in a device status word that
 *    sp_check_status() reads.
 *  - Microphone pairs p = (i, j), i < j, are numbered in the order of Eq. 7:
 *    (0,1), (0,2), ..., (M-2, M-1).  B = N/2 + 1 frequency bins k = 0..N/2 and
 *    L = P * B.  STFT frames are [T][M][B] complex64 (interleaved float re, im).
 *  - A spectrum entry with |X|^2 < 1e-30 counts as zero; every cross spectrum using it
 *    is 0 (Eq. 3 divides by magnitudes).  Argmax ties go to the lowest index; a frame
 *    whose every score is NaN gets index -1.
 *  - Handles are not thread-safe: calls that use the same handle from several host
 *    threads, or on several streams at once, must be serialised by the caller
 *    (a handle owns one device workspace that every localize call on it reuses).
 */
#ifndef SVDPHAT_H
#define SVDPHAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SP_OK        0
#define SP_EINVAL   (-1)  /* bad argument (size, null pointer, misaligned pointer, ...)   */
#define SP_ENOMEM   (-2)  /* device or host allocation failed                             */
#define SP_ECUDA    (-3)  /* a CUDA runtime/driver call failed                            */
#define SP_ETIMEOUT (-4)  /* a bounded device wait gave up (see sp_check_status)          */
#define SP_ENOTIMPL (-5)  /* combination of mode / precision / size not supported         */
#define SP_EBOUNDS  (-6)  /* debug build only: a device bounds check failed (see sp_check_status) */

typedef enum {
    SP_MODE_SRP = 0,             /* Eq. 9 + Eq. 6: argmax Re{W X} over all Q rows           */
    SP_MODE_SVD_EXHAUSTIVE = 1,  /* Eq. 12 + Eq. 14: argmax Re{D Z}, Z = V^H X              */
    SP_MODE_SVD_KDTREE = 2,      /* Eq. 15: nearest normalised row D^_q to conj(Z/||Z||)    */
    SP_MODE_SVD_LEARNED = 3      /* Eq. 14 over the cells a trained network proposes: needs a
                                    proposal handle, so it runs through sp_localize_learned;
                                    sp_localize and the batch calls reject it (SP_EINVAL)     */
} sp_mode;

typedef enum {
    SP_PREC_FP32 = 0,  /* FP32 SIMT arithmetic throughout                                    */
    SP_PREC_FP16 = 1,  /* FP16 tensor-core projections, FP32 accumulate, FP32 rescoring of a candidate window */
    SP_PREC_BF16 = 2   /* BF16 tensor-core projections, FP32 accumulate, FP32 rescoring of a candidate window */
} sp_prec;

typedef struct sp_steering sp_steering;  /* TDOA table + steering matrix W (Eq. 2, 4, 8) */
typedef struct sp_basis sp_basis;        /* rank-K basis V, D = U S, D^, k-d tree (Eq. 10-15) */
typedef struct sp_proposal sp_proposal;  /* learned cell proposal over a basis (no counterpart in the paper) */
typedef struct sp_batch sp_batch;        /* many streams in one CUDA-graph launch (no counterpart in the paper) */

/* Thread-local message describing the last failure of this thread (never NULL). */
const char *sp_last_error(void);

/* Library version as 10000*major + 100*minor + patch. */
int sp_version(void);

/* ---------------------------------------------------------------------------------
 * Offline step 1 of Algorithm 1: steering (Eq. 2, Eq. 4, Eq. 8).
 *
 * mic_xyz: host, M x 3 doubles (metres), M in [2, 64].
 * dirs:    host, Q x 3 doubles; candidate directions s_q (need not be unit length,
 *          Eq. 2 divides by ||s_q||; a zero vector is SP_EINVAL).  Q in [1, 2^24].
 * fs, c:   sample rate (Hz) and speed of sound (m/s), both > 0.
 * N:       STFT frame size, even, in [4, 8192].
 * flags:   bit 0 (SP_STEER_MATERIALIZE_W): also materialise W (Q x L complex64 on the
 *          device) for SP_MODE_SRP.  Without it SRP localisation is SP_ENOTIMPL.
 * out:     receives the new handle.
 *
 * The TDOA table tau[q][p] = fs/c * (r_j - r_i) . s_q/||s_q|| is computed on the device
 * in FP64 with the fixed operation order n = sqrt((sx*sx + sy*sy) + sz*sz),
 * u = s / n, tau = (fs/c) * ((dx*ux + dy*uy) + dz*uz), every step correctly rounded.
 * W[q][p*B + k] = exp(2 pi i k tau[q][p] / N), phase reduced in FP64.
 * Synchronous (returns when the table is built).
 * --------------------------------------------------------------------------------- */
#define SP_STEER_MATERIALIZE_W 1
int sp_build_steering(const double *mic_xyz, int M, const double *dirs, int Q,
                      double fs, double c, int N, int flags, sp_steering **out);

/* The same offline step for sources at given positions (the near field, Eq. 1; Section 2
 * gives Eq. 2 as its limit for a source far from a small array, and Section 6 names the
 * near-field effect as an extension):
 *   tau[q][p] = fs/c * (||s_q - r_i|| - ||s_q - r_j||),  pair p = (i, j), i < j,
 * with src_xyz the Q x 3 candidate source positions in metres, in the microphones'
 * frame.  Computed on the device in FP64 with every norm in the fixed order
 * sqrt((ex*ex + ey*ey) + ez*ez), e = s - r, then tau = (fs/c) * (n_i - n_j), each step
 * correctly rounded.  Everything downstream (W, direction classes, sp_svd_reduce, every
 * sp_localize mode, step 4 with d_m = -fs/c ||s_q - r_m||) is the same as for directions.
 * A source at the coordinate origin is SP_EINVAL (s_q / ||s_q|| is the direction used to
 * assign learned-proposal cells); other arguments and errors as for sp_build_steering.
 * sp_steering_nearfield reports which builder made a handle (1 near field, 0 directions). */
int sp_build_steering_nearfield(const double *mic_xyz, int M, const double *src_xyz, int Q,
                                double fs, double c, int N, int flags, sp_steering **out);
int sp_steering_nearfield(const sp_steering *st, int *nearfield);

/* Dimensions of a steering handle; any pointer may be NULL. */
int sp_steering_dims(const sp_steering *st, int *M, int *P, int *Q, int *N, int *B);

/* Direction classes: q and q' are one class when max_p |tau[q][p] - tau[q'][p]| <= 1e-9
 * samples; their rows of W (Eq. 8) are then identical, so every SRP-PHAT or SVD-PHAT
 * score is the same for both (a line array cannot tell directions on a cone apart, a
 * planar array mirror images).  The SVD-PHAT searches evaluate each class once, at its
 * lowest index, so they return the lowest index of the winning class.
 * n_classes (may be NULL) receives the number of classes; rep_of_host (Q int32, may be
 * NULL) receives, for every q, the lowest index of its class. */
int sp_steering_classes(const sp_steering *st, int *n_classes, int32_t *rep_of_host);

/* Copy the FP64 TDOA table (Q x P, row-major) to host memory. Synchronous. */
int sp_steering_tau(const sp_steering *st, double *tau_host);

/* Copy W (Q x L complex64, row-major, column p*B + k as in Eq. 8) into a device buffer.
 * SP_EINVAL if W was not materialised. Asynchronous on stream. */
int sp_steering_w(const sp_steering *st, void *w_dev, void *stream);

void sp_steering_destroy(sp_steering *st);

/* ---------------------------------------------------------------------------------
 * Offline steps 2-4 of Algorithm 1 (Eq. 10-13, Section 3).
 *
 * Truncated SVD W ~= U S V^H by randomized block subspace iteration in FP64 on the
 * device (products with W generated from the TDOA table) and a Rayleigh-Ritz step on
 * the host.  K is the smallest rank with sum_{k<=K} s_k^2 >= (1 - delta) Tr{W W^H}
 * (Eq. 11, Tr{W W^H} = Q L); if that K splits a cluster of equal singular values
 * (s_{K+1}^2 >= s_K^2 - 1e-10 s_1^2) it is extended to the end of the cluster.
 * D = U S = W V (Eq. 13) is formed in FP64, D^_q = D_q / ||D_q||, and a k-d tree over
 * the real 2K-dimensional rows [Re D^_q, Im D^_q] is built on the host and uploaded.
 *
 * delta in (0, 1).  flags: reserved, pass 0.  K_out (may be NULL) receives K.
 * The steering handle must outlive the basis.  Synchronous.
 * --------------------------------------------------------------------------------- */
int sp_svd_reduce(const sp_steering *st, double delta, int flags, sp_basis **out, int *K_out);

/* K, the number of computed Ritz values n_sigma, and (if sigma2_host != NULL) the
 * first min(n_sigma, cap) squared singular values in descending order. */
int sp_basis_info(const sp_basis *b, int *K, int *n_sigma, double *sigma2_host, int cap);

/* Copy V (L x K complex128, row-major, interleaved re/im) or D (Q x K complex128) to host. */
int sp_basis_v(const sp_basis *b, double *v_host);
int sp_basis_d(const sp_basis *b, double *d_host);

/* k-d tree shape: number of nodes, leaf bucket size and depth. */
int sp_basis_kdtree_info(const sp_basis *b, int *n_nodes, int *leaf_size, int *depth);

void sp_basis_destroy(sp_basis *b);

/* ---------------------------------------------------------------------------------
 * Persistence of the offline phase (Algorithm 1, offline steps 1-3): the array geometry
 * and grid that define W (Eq. 2, 4), the rank K of Eq. 11, V and D = U S (Eq. 12, 13).
 *
 * sp_save_basis writes b to path (a new file, or overwritten): a little-endian binary
 * with an 80-byte header (magic "SVDPHAT1", version 1, M, Q, N, K, number of singular
 * values, the steering model (0 directions, 1 source positions), fs, c, delta), the FP64
 * arrays mic [M][3], dirs or source positions [Q][3], sigma^2, V [L][K] and
 * D [Q][K] (complex as re, im pairs), and an FNV-1a 64 checksum of all preceding bytes.
 * Returns SP_EINVAL if the file cannot be opened or written.
 *
 * sp_load_basis reads such a file, rebuilds the steering handle with the builder of its
 * model (flags as in sp_build_steering: SP_STEER_MATERIALIZE_W or 0), the device operands
 * and the k-d tree on the current device, and returns a basis that OWNS its steering handle (released by
 * sp_basis_destroy; obtain it with sp_basis_steering, never destroy it separately).
 * Results through a loaded basis are bit-identical to those through the saved one.
 * A malformed file (wrong magic or version, sizes out of range, a length that does not
 * match the header, a checksum mismatch, non-finite values) gives SP_EINVAL before any
 * device work; *out is NULL on every error.  K_out may be NULL.
 *
 * sp_basis_steering returns the steering handle a basis was built on (borrowed: valid
 * while the basis lives).
 * --------------------------------------------------------------------------------- */
int sp_save_basis(const sp_basis *b, const char *path);
int sp_load_basis(const char *path, int flags, sp_basis **out, int *K_out);
int sp_basis_steering(const sp_basis *b, const sp_steering **out);

/* ---------------------------------------------------------------------------------
 * Online step 1 (Eq. 3, Eq. 7) on its own: PHAT cross spectra of all pairs.
 * frames_dev: device [T][M][B] complex64 (8-byte aligned).  x_dev: device [T][L]
 * complex64, column p*B + k.  T >= 0 (T = 0 is a no-op).
 * --------------------------------------------------------------------------------- */
int sp_phat(const void *frames_dev, int T, int M, int B, void *x_dev, void *stream);

/* ---------------------------------------------------------------------------------
 * Online steps 1-2 (Eq. 3, 7, 12): Z = V^H X for every frame, PHAT fused.
 * z_dev: device [T][K] complex64.  prec selects FP32 SIMT or the FP16/BF16 tensor-core
 * GEMM (FP32 accumulate).
 * --------------------------------------------------------------------------------- */
int sp_project(const sp_basis *b, const void *frames_dev, int T, sp_prec prec,
               void *z_dev, void *stream);

/* ---------------------------------------------------------------------------------
 * The online hot path (Algorithm 1, online steps 1-4) for T frames.
 *
 * mode SP_MODE_SRP:            idx = argmax_q Re{W_q X} (needs a materialised W; prec
 *                              must be SP_PREC_FP32).
 * mode SP_MODE_SVD_EXHAUSTIVE: idx = argmax_q Re{D_q Z} (Eq. 14).  With FP16/BF16 the
 *                              reduced-precision scan collects, per frame, every class
 *                              whose score lies within the scan's rounding bound of the
 *                              frame's maximum and rescores them in FP32 against FP32 Z
 *                              and D; a frame with more than 14 such classes is scored in
 *                              FP32 against every class instead.  Either way the result
 *                              equals an FP32 scan of the same Z (up to FP32 summation
 *                              order).
 * mode SP_MODE_SVD_KDTREE:     idx = nearest D^_q to conj(Z/||Z||) by exact k-d tree
 *                              search (Eq. 15), FP32 distances.
 *
 * idx_dev:        device int32 [T], required.
 * score_dev:      device float [T] or NULL: Y_idx = Re{W_idx X}, the SRP-PHAT energy of
 *                 the chosen direction from its regenerated row of W (Algorithm 1,
 *                 online step 4).  NULL skips step 4.
 * proj_score_dev: device float [T] or NULL: the search's own score, Re{D_idx Z} for the
 *                 SVD modes (Re{D^_idx Z^} for the k-d tree), Re{W_idx X} for SRP.
 * Asynchronous on stream; the basis workspace is reused by the next call.
 *
 * Frame alignment: frames must be 8-byte aligned.  For 7-microphone arrays the FP16/BF16
 * path reads 16-byte-aligned frame buffers with TMA (the fast GEMM1 kernel); a buffer 8 bytes
 * off a 16-byte boundary runs a register-fed GEMM1 whose FP32 summation order differs, so
 * scores can differ in the last bits (and an index only where two scores tie that closely).
 * Results are bit-identical between calls on buffers of the same alignment.
 * --------------------------------------------------------------------------------- */
int sp_localize(const sp_basis *b, const void *frames_dev, int T, sp_mode mode, sp_prec prec,
                int32_t *idx_dev, float *score_dev, float *proj_score_dev, void *stream);

/* ---------------------------------------------------------------------------------
 * Online step 3 by the k-d tree (Eq. 15) on its own, from given projections: z_dev is device
 * [T][K] complex64 (Z of Eq. 12, e.g. from sp_project).  idx_dev (device int32 [T]) receives
 * the nearest normalised row D^_q to conj(Z / ||Z||) (exact search, FP32 distances, ties to
 * the lowest index; -1 where ||Z|| is 0 or not finite) and proj_dev (device float [T] or NULL)
 * the score Re{D^_idx Z^} = 1 - d^2 / 2.  visits_dev (device int32 [T][2] or NULL) receives per
 * query the tree nodes and the leaf buckets (32 points each) the search visited.  The tree's
 * nodes are read from shared memory when they fit in 96 KB.  Asynchronous on stream.
 * --------------------------------------------------------------------------------- */
int sp_kdtree_search(const sp_basis *b, const void *z_dev, int T, int32_t *idx_dev, float *proj_dev,
                     int32_t *visits_dev, void *stream);

/* Plain SRP-PHAT (Eq. 5, 6, 9) straight from a steering handle (no basis needed). */
int sp_localize_srp(const sp_steering *st, const void *frames_dev, int T,
                    int32_t *idx_dev, float *score_dev, void *stream);

/* ---------------------------------------------------------------------------------
 * sp_localize from HOST buffers: frames_host [T][M][B] complex64, idx_host int32 [T],
 * score_host / proj_score_host float [T] or NULL.  Frames are copied in chunks of
 * chunk_frames (0 = library default) through two device staging buffers so that the
 * host-to-device copy of chunk c+1 overlaps the localisation of chunk c.  Pinned host
 * memory is needed for the copies to be asynchronous.  Returns when every result is
 * in host memory.
 * --------------------------------------------------------------------------------- */
int sp_localize_host(const sp_basis *b, const void *frames_host, int T, sp_mode mode,
                     sp_prec prec, int32_t *idx_host, float *score_host,
                     float *proj_score_host, int chunk_frames, void *stream);

/* ---------------------------------------------------------------------------------
 * sp_localize without any allocation (the paper has no counterpart; this is a deployment
 * aid).  Some callers cannot call cudaMalloc on their processing path: real-time audio
 * callbacks and plugin hosts, where the allocator can block on driver locks and miss the
 * audio deadline, and deployments whose device memory budget is fixed at start-up.  This
 * entry point runs the same kernels as sp_localize with SP_MODE_SVD_EXHAUSTIVE, but keeps
 * its scratch (the Z vectors and their norms) in an 8 MiB array compiled into the library,
 * which every GPU that loads the library holds until the process exits.
 *
 * prec: SP_PREC_FP16 or SP_PREC_BF16 (SP_ENOTIMPL otherwise).  A call needs
 * about T * (8 K + 16) bytes of that scratch (K from sp_svd_reduce; at K = 48 that is up to
 * 20,900 frames per call); larger T is rejected with SP_EINVAL before any work is queued.
 * idx_dev, score_dev, proj_score_dev: as for sp_localize.  The caller still provides the
 * frames and all outputs.
 *
 * Arguments are checked as in sp_localize (SP_EINVAL for a NULL or misaligned pointer, T < 0
 * or T > 2^28), and a basis without a tensor-core plan (2K > 288) gives SP_ENOTIMPL.
 *
 * Warm-up: the first call on a device looks up the array's device address (with that
 * device current) and caches it, and the first launch of each kernel loads it and sets its
 * shared-memory limit.  A call with T == 0 does all of this and launches nothing: make one
 * such call per device and basis, outside the processing path and before any stream
 * capture.  After it, calls allocate nothing (no cudaMalloc, cudaFree or allocating
 * library routine).  Every call on a device shares the one array, which keeps the last
 * call's contents; nothing in it needs to start at zero.  Calls whose work overlaps on the
 * GPU (other streams, other threads) race on the array: serialise them. */
int sp_localize_noalloc(const sp_basis *b, const void *frames_dev, int T, sp_prec prec,
                        int32_t *idx_dev, float *score_dev, float *proj_score_dev, void *stream);

/* ---------------------------------------------------------------------------------
 * The STFT front end of Section 2 (the expression X_m^l[k] that Eq. 3 starts from) and the
 * binary time-frequency mask the paper's conclusion proposes.
 *
 * sp_stft: X_m^l[k] = sum_{n<N} w[n] x_m[l hop + n] exp(-2 pi i k n / N) for k = 0 .. N/2 and
 * every whole frame l = 0 .. T-1, T = floor((n_samples - N) / hop) + 1 (0 when n_samples < N),
 * with the sine window w[n] = sin(pi (n + 1/2) / N) and no normalisation.  FP32 arithmetic:
 * an N/2-point complex FFT of the even/odd samples (radix-2, shared memory) and the real-input
 * post-processing.
 *   samples_dev: device float [M][ld] (channel rows, 4-byte aligned), n_samples <= ld per row.
 *   N: power of two in [4, 8192]; hop >= 1.
 *   mask_dev: device uint8 [T][N/2+1] or NULL; a bin whose mask is 0 is written as 0 for every
 *     channel.  Under Eq. 3's zero rule such a bin contributes nothing to any cross spectrum,
 *     so it drops out of Eq. 5, 9, 12, 14 and of online step 4.
 *   frames_dev: device [T][M][N/2+1] complex64 (8-byte aligned), the layout sp_localize takes.
 *   T_out (may be NULL) receives T.  Errors: SP_EINVAL (sizes, pointers), SP_ENOTIMPL (N).
 * sp_apply_mask: out[l][m][k] = mask[l][k] ? frames[l][m][k] : 0 for STFT frames from elsewhere
 *   ([T][M][B] complex64, 8-byte aligned; out may equal frames).
 * sp_localize_samples: sp_stft of the first T frames into the basis's workspace (M and N of the
 *   basis), then sp_localize of those frames; T <= the whole frames in the samples.  Outputs,
 *   modes, precisions and errors as for sp_localize.  Asynchronous on stream.
 * --------------------------------------------------------------------------------- */
int sp_stft(const float *samples_dev, int M, long long n_samples, long long ld, int N, int hop,
            const uint8_t *mask_dev, void *frames_dev, int *T_out, void *stream);
int sp_apply_mask(const void *frames_dev, int T, int M, int B, const uint8_t *mask_dev, void *out_dev,
                  void *stream);
int sp_localize_samples(const sp_basis *b, const float *samples_dev, long long n_samples, long long ld, int hop,
                        const uint8_t *mask_dev, int T, sp_mode mode, sp_prec prec, int32_t *idx_dev,
                        float *score_dev, float *proj_score_dev, void *stream);

/* ---------------------------------------------------------------------------------
 * The energy-weighted DOA error of Section 4 (Eq. 16-20) for the T frames of one
 * configuration: RMSE_alpha = || sum_l f_alpha(s_idx[l]) Y[l] / sum_l Y[l] - f_alpha(s0) ||_2,
 * with s_idx[l] the unit direction of grid point idx[l] of st, Y = score_dev (the energy of the
 * chosen direction, Algorithm 1's online step 4 as sp_localize writes it), and f_1 (arc, Eq. 16,
 * 17), f_2 (upper hemisphere, Eq. 18), f_3 (identity, Eq. 19) for the 1-D, 2-D and 3-D arrays.
 * Frames with idx < 0 or a non-finite Y are left out.  FP64 sums in a fixed order.
 * idx_dev: device int32 [T]; score_dev: device float [T]; s0: host double [3], the true
 * direction (need not be unit length); alpha in {1, 2, 3}; rmse_out: host double.
 * Synchronous on stream (allocates 32 bytes of device memory).  Errors: SP_EINVAL (arguments,
 * energies summing to zero), SP_ECUDA.
 * --------------------------------------------------------------------------------- */
int sp_weighted_doa_error(const sp_steering *st, const int32_t *idx_dev, const float *score_dev, int T,
                          const double *s0, int alpha, double *rmse_out, void *stream);

/* Synchronise stream and report a device-side failure recorded since the last call
 * (SP_ETIMEOUT if a bounded wait gave up; SP_EBOUNDS if, in the SP_DEBUG build
 * libsvdphat_debug.so, a device bounds check failed and its access was skipped), clearing it. */
int sp_check_status(void *stream);

/* Measurement aid (the paper has no counterpart): the FP32 fused multiply-add rate of the
 * current device in TFLOP/s (2 flops per FMA), from a kernel of independent FMA chains on
 * every SM, timed with CUDA events.  It is the denominator of the plain FP32 SRP-PHAT roofline
 * (Eq. 9 costs 4 Q L flops per frame).  Synchronous; allocates 2 KB of device memory. */
int sp_fp32_fma_peak(double *tflops);

/* For tests: set the iteration budget of every bounded device wait (0 = default).
 * A budget of 1 makes waits give up at once, which exercises SP_ETIMEOUT. */
int sp_set_wait_budget(long long iterations);

/* =================================================================================
 * Batched localisation (no counterpart in the paper, whose Algorithm 1 handles one stream
 * of frames): n independent streams, each with its own basis (array, grid, N, K), frames
 * and frame count, localised by one CUDA-graph launch whose branches run concurrently.
 * Each stream computes exactly what sp_localize computes for it (same kernels, same
 * results); where a basis has no tensor-core path (2K > 288 or M > 16) an FP16/BF16 request
 * runs that stream in FP32.
 *
 * sp_batch_create: bases[i] (must outlive the plan), frames_dev[i] (device [T[i]][M][B]
 * complex64, the caller's buffer, read at every run), T[i] >= 1, mode and prec as in
 * sp_localize, idx_dev[i] / score_dev[i] / proj_dev[i] as in sp_localize (score_dev and
 * proj_dev may be NULL arrays or hold NULL entries).  Shapes and pointers are fixed for the
 * plan's lifetime.  Synchronous: after the work already queued on `stream` (which may be
 * writing the frames), it runs every stream once (sizing the workspaces), then captures the
 * graph; with SP_BATCH_AUTOTUNE it builds and times the candidate launch
 * shapes (branches in {8, 32, 128, n} x tiles per GEMM1 CTA in {1, 2, 4}; with
 * SP_BATCH_TUNE_KERNELS also x GEMM1 kernel: TMA-fed where it applies or register-fed,
 * the latter tried only when some stream could use either) and keeps the fastest.  Without
 * SP_BATCH_TUNE_KERNELS every stream's results are bit-identical to sp_localize's; with it,
 * a 7-microphone stream may take the register-fed GEMM1, whose FP32 sums run in another
 * order (its results then equal sp_localize's on a frame buffer 8 bytes off a 16-byte
 * boundary, which takes that kernel).  With a tune cache set (sp_set_tune_cache), an
 * autotuned plan first looks up the batch's signature (device, mode, precision, every
 * stream's M, B, K, class count, T and precision) and, if present, takes that shape without
 * measuring; otherwise it measures and stores the winner.  Errors: SP_EINVAL (bad
 * arguments, per stream as sp_localize; a tune cache that exists but does not parse), SP_ECUDA.
 * sp_batch_run: one graph launch on stream (asynchronous).
 * sp_batch_info: the chosen shape (proj_variant 0: TMA-fed GEMM1 where it applies, 1:
 * register-fed; grouped 1: the groups below are localised one call each), the measured
 * milliseconds of one launch (autotuned plans, else 0), how many streams run in FP32, whether
 * the shape came from the tune cache, and how many groups the plan formed.  Any out pointer
 * may be NULL.
 * Groups: streams with the same basis and precision whose frames start on a 16-byte boundary
 * (at most 2^28 frames per group) form a group.  A grouped plan copies a group's frames into
 * one buffer the plan owns, runs one sp_localize-equivalent call on it and copies the results
 * back to each stream's outputs: the same kernels on the same frames, so every stream's
 * results stay bit-identical to its own sp_localize call, while the GPU sees a few large
 * launches instead of many small ones.  The plan holds the copy (as many bytes as the grouped
 * streams' frames).  Autotuned plans try both forms; other plans group only with
 * SP_BATCH_GROUP.  (On the bench's mix of 256 streams of 50-2000 frames over 16 bases the
 * per-stream form was the faster: the copies cost more than the launches they save.)
 * sp_localize_batched: create (no autotuning), run once, synchronise, destroy.
 * ================================================================================= */
#define SP_BATCH_AUTOTUNE 1
#define SP_BATCH_TUNE_KERNELS 2
#define SP_BATCH_GROUP 4
int sp_batch_create(int n, const sp_basis *const *bases, const void *const *frames_dev, const int *T,
                    sp_mode mode, sp_prec prec, int32_t *const *idx_dev, float *const *score_dev,
                    float *const *proj_dev, int flags, void *stream, sp_batch **out);
int sp_batch_run(sp_batch *bt, void *stream);
int sp_batch_info(const sp_batch *bt, int *branches, int *tiles_per_cta, int *proj_variant, float *ms,
                  int *n_fp32, int *from_cache, int *grouped, int *n_groups);
void sp_batch_destroy(sp_batch *bt);
int sp_localize_batched(int n, const sp_basis *const *bases, const void *const *frames_dev, const int *T,
                        sp_mode mode, sp_prec prec, int32_t *const *idx_dev, float *const *score_dev,
                        float *const *proj_dev, void *stream);

/* The autotune cache (host only; no device call): path of a JSON file holding
 * {"format": "svdphat-tune-cache", "version": 1, "plans": {key: {"branches": b,
 * "tiles_per_cta": t, "proj_variant": v, "grouped": g, "ms": m}}} ("grouped" may be absent:
 * 0); NULL or "" disables it (the default).
 * The file is created on the first store and rewritten whole through a temporary file and
 * a rename; a file that exists but does not parse is never overwritten (SP_EINVAL).
 * sp_tune_cache_get: *found = 1 and the stored shape if key is present, else *found = 0
 * (out pointers other than found may be NULL).  sp_tune_cache_put: stores or replaces an
 * entry (branches >= 1, tiles_per_cta in {1, 2, 4}, proj_variant in {0, 1}, grouped in {0, 1},
 * ms >= 0).
 * Keys: 1-512 printable ASCII characters without '"' or '\'.  Errors: SP_EINVAL. */
int sp_set_tune_cache(const char *path);
int sp_tune_cache_get(const char *key, int *branches, int *tiles_per_cta, int *proj_variant, float *ms,
                      int *grouped, int *found);
int sp_tune_cache_put(const char *key, int branches, int tiles_per_cta, int proj_variant, float ms, int grouped);

/* =================================================================================
 * Learned direction proposal (no counterpart in the paper).  The paper searches Eq. 14
 * exhaustively or by the k-d tree of Eq. 15 (Section 3).  This search lets a small
 * network propose coarse cells of the direction grid and evaluates Eq. 14 only over the
 * directions of those cells, in FP32; frames the network is unsure of take the exhaustive
 * scan.  Definitions:
 *   cell of direction q: the cell direction with the largest dot product with q (after
 *     normalising both); dot products within 1e-12 of the largest tie, lowest cell wins.
 *   features of a frame: x = [Re Z_0, Im Z_0, Re Z_1, Im Z_1, ...] / ||Z||, F = 2K reals
 *     (Z of Eq. 12; x = 0 when ||Z|| = 0).
 *   network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), logits = W3 h2 + b3.
 *   parameters (FP32, flat, in this order): W1 [H1][F], b1 [H1], W2 [H2][H1], b2 [H2],
 *     W3 [C][H2], b3 [C], all row-major.
 *   loss: mean over the batch of -log softmax(logits)[label]; a label outside [0, C)
 *     contributes nothing.  Training label: the cell of the frame's Eq. 14 argmax.
 *   optimiser: Adam (Kingma & Ba, 2015) with beta1 0.9, beta2 0.999, eps 1e-8.
 * All device pointers are caller-owned; calls are asynchronous on `stream` unless noted.
 * ================================================================================= */

/* Create a proposal for basis b (which must outlive it): C cell directions cell_dirs
 * [C][3] (host, need not be unit length), hidden sizes H1, H2 (multiples of 64 in
 * [64, 256]), 1 <= C <= 4096, 2K <= 288 (the tensor-core plan of GEMM1).  Weights are drawn uniformly in
 * +-sqrt(6 / fan_in) from a counter-based generator keyed by seed; biases are 0.
 * Synchronous.  Errors: SP_EINVAL (bad arguments), SP_ENOTIMPL (2K > 288). */
int sp_proposal_create(const sp_basis *b, const double *cell_dirs, int C, int H1, int H2,
                       unsigned long long seed, sp_proposal **out);
void sp_proposal_destroy(sp_proposal *p);
int sp_proposal_dims(const sp_proposal *p, int *F, int *H1, int *H2, int *C, long long *n_params);
/* cell_of_host: int32 [Q], the cell of every grid direction. */
int sp_proposal_cells(const sp_proposal *p, int32_t *cell_of_host);
/* Copy the FP32 parameters to / from host memory (n_params floats).  Synchronous;
 * setting also resets the Adam state.  Non-finite values give SP_EINVAL. */
int sp_proposal_get_params(const sp_proposal *p, float *host);
int sp_proposal_set_params(sp_proposal *p, const float *host);

/* Training examples from T frames (device [T][M][B] complex64): x_dev float [T][F], the
 * features of Z (FP16/BF16 tensor-core or FP32 projection per prec), and label_dev int32
 * [T], the cell of the exhaustive Eq. 14 argmax (-1 for a frame without one). */
int sp_proposal_examples(const sp_proposal *p, const void *frames_dev, int T, sp_prec prec,
                         float *x_dev, int32_t *label_dev, void *stream);

/* FP32 forward pass of n feature rows x_dev [n][F] -> logits_dev float [n][C]. */
int sp_proposal_forward_f32(const sp_proposal *p, const float *x_dev, int n, float *logits_dev,
                            void *stream);
/* Loss (loss_dev: one float, or NULL) and its gradient grad_dev (float [n_params], the
 * parameter layout) over n rows, FP32.  Does not change the parameters. */
int sp_proposal_grad(const sp_proposal *p, const float *x_dev, const int32_t *label_dev, int n,
                     float *grad_dev, float *loss_dev, void *stream);
/* One Adam step on the batch: rows x_dev[rows_dev[i]] (rows_dev int32 [n]) or, with
 * rows_dev NULL, the first n rows.  lr > 0.  loss_dev as above (before the step). */
int sp_proposal_train_step(sp_proposal *p, const float *x_dev, const int32_t *label_dev,
                           const int32_t *rows_dev, int n, float lr, float *loss_dev, void *stream);

/* Tensor-core inference of the network (BF16 weights and activations, FP32 accumulate)
 * from Z (device [T][K] complex64) and ||Z||^2 (device float [T]): top_dev int32 [T][8],
 * the 8 cells with the largest logits (largest first, ties -> lowest cell), conf_dev float
 * [T], the largest softmax probability, and logits_dev float [T][C] or NULL. */
int sp_proposal_infer(const sp_proposal *p, const void *z_dev, const float *zn2_dev, int T,
                      float *logits_dev, int32_t *top_dev, float *conf_dev, void *stream);

/* The learned search (Algorithm 1 online steps 1-4 with the proposal in step 3): PHAT and
 * Z = V^H X on the tensor cores (prec SP_PREC_FP16 or SP_PREC_BF16), the network, then
 * argmax Re{D_q Z} in FP32 over the directions of the n_top (1..8) proposed cells; a frame
 * whose largest softmax probability is not >= theta takes the exhaustive scan of
 * sp_localize (SP_MODE_SVD_EXHAUSTIVE).  idx_dev, score_dev, proj_score_dev as in
 * sp_localize (idx is the lowest index of the winning direction class); fallback_dev
 * int32 [T] or NULL receives 1 for frames that fell back, else 0. */
int sp_localize_learned(const sp_proposal *p, const void *frames_dev, int T, sp_prec prec,
                        int n_top, float theta, int32_t *idx_dev, float *score_dev,
                        float *proj_score_dev, int32_t *fallback_dev, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SVDPHAT_H */
