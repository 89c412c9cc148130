// Offline steps 2-3 of Algorithm 1: truncated SVD of the steering matrix W (Eq. 10),
// rank K from the trace rule (Eq. 11), D = U S = W V (Eq. 13).
//
// Method: randomized block subspace iteration (Halko, Martinsson & Tropp, SIAM Review
// 2011, Algorithm 4.4) with a Rayleigh-Ritz step.  Products with W (Q x L) and W^H run in
// FP64 on the device; W is regenerated from the TDOA table into an FP64 buffer that lives
// only for the duration of the call.  Orthonormalisation (modified Gram-Schmidt, applied
// twice) and the small r x r Hermitian eigenproblem (cyclic Jacobi) run on the host.
//
//   Omega: L x r complex Gaussian
//   Y = W Omega;  repeat n_power times { Y = orth(Y); H = orth(W^H Y); Y = W H }
//   Y = orth(Y);  Bh = W^H Y (= B^H, B = Y^H W, r x L)
//   B B^H = Bh^H Bh = U~ S^2 U~^H  ->  sigma_k^2, V = Bh U~ S^-1
// K = smallest k with sum_{j<=k} sigma_j^2 >= (1 - delta) Q L (Tr{W W^H} = Q L exactly,
// every entry of W has unit modulus), extended over a cluster of equal singular values;
// if K comes too close to r the block is doubled and the iteration restarted.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <random>
#include <vector>

#include "common.h"

namespace sp {

using cd = std::complex<double>;

// W[q][l] = exp(2 pi i k tau[q][p] / N), l = p*B + k, FP64 (the phase reduced in FP64).
__global__ void w64_kernel(const double *__restrict__ tau, int Q, int P, int B, int N,
                           double2 *__restrict__ W) {
    const long long L = (long long)P * B;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)Q * L) return;
    const long long q = idx / L;
    const int l = (int)(idx % L);
    const int p = l / B, k = l % B;
    const double turns = (double)k * tau[q * P + p] / (double)N;
    const double r = turns - rint(turns);
    double s, c;
    sincospi(2.0 * r, &s, &c);
    W[idx] = make_double2(c, s);
}

// C (m x n) = op(A) B, op(A) = A (m x kk, row-major, lda) or A^H (A stored kk x m).
// B is kk x n row-major.  16 x 16 output tile per block, one output per thread.
__global__ void zgemm_kernel(int conjA, int m, int n, int kk, const double2 *__restrict__ A,
                             long long lda, const double2 *__restrict__ B, long long ldb,
                             double2 *__restrict__ C, long long ldc) {
    __shared__ double2 As[16][17];
    __shared__ double2 Bs[16][17];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const long long row = (long long)blockIdx.y * 16 + ty;
    const long long col = (long long)blockIdx.x * 16 + tx;
    double cr = 0.0, ci = 0.0;
    for (int k0 = 0; k0 < kk; k0 += 16) {
        // As[ty][tx] = op(A)[blockrow + ty][k0 + tx]
        {
            const long long r = (long long)blockIdx.y * 16 + ty;
            const long long k = k0 + tx;
            double2 v = make_double2(0.0, 0.0);
            if (r < m && k < kk) {
                if (conjA) {
                    v = A[k * lda + r];
                    v.y = -v.y;
                } else {
                    v = A[r * lda + k];
                }
            }
            As[ty][tx] = v;
        }
        {
            const long long k = k0 + ty;
            Bs[ty][tx] = (k < kk && col < n) ? B[k * ldb + col] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const double2 a = As[ty][j], b = Bs[j][tx];
            cr = fma(a.x, b.x, cr);
            cr = fma(-a.y, b.y, cr);
            ci = fma(a.x, b.y, ci);
            ci = fma(a.y, b.x, ci);
        }
        __syncthreads();
    }
    if (row < m && col < n) C[row * ldc + col] = make_double2(cr, ci);
}

static int zgemm(bool conjA, int m, int n, int kk, const void *A, long long lda, const void *B,
                 long long ldb, void *C, long long ldc) {
    dim3 blk(16, 16), grd((n + 15) / 16, (m + 15) / 16);
    zgemm_kernel<<<grd, blk>>>(conjA ? 1 : 0, m, n, kk, (const double2 *)A, lda, (const double2 *)B,
                               ldb, (double2 *)C, ldc);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

// ------------------------------------------------------------------ host linear algebra
// Columns of the row-major n x r matrix Y made orthonormal in place by modified
// Gram-Schmidt applied twice; a column that collapses is replaced by a random vector.
static void orthonormalize(std::vector<cd> &Y, int n, int r, std::mt19937_64 &rng) {
    std::normal_distribution<double> nd;
    std::vector<cd> C((size_t)n * r);  // column-major copy
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < r; ++j) C[(size_t)j * n + i] = Y[(size_t)i * r + j];
    for (int j = 0; j < r; ++j) {
        cd *col = &C[(size_t)j * n];
        double n0 = 0;
        for (int i = 0; i < n; ++i) n0 += std::norm(col[i]);
        n0 = std::sqrt(n0);
        for (int attempt = 0; attempt < 3; ++attempt) {
            for (int pass = 0; pass < 2; ++pass)
                for (int c = 0; c < j; ++c) {
                    const cd *qc = &C[(size_t)c * n];
                    cd d = 0;
                    for (int i = 0; i < n; ++i) d += std::conj(qc[i]) * col[i];
                    for (int i = 0; i < n; ++i) col[i] -= d * qc[i];
                }
            double nn = 0;
            for (int i = 0; i < n; ++i) nn += std::norm(col[i]);
            nn = std::sqrt(nn);
            if (nn > 1e-13 * n0 && nn > 0) {
                for (int i = 0; i < n; ++i) col[i] /= nn;
                break;
            }
            for (int i = 0; i < n; ++i) col[i] = cd(nd(rng), nd(rng));
            n0 = 0;
            for (int i = 0; i < n; ++i) n0 += std::norm(col[i]);
            n0 = std::sqrt(n0);
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < r; ++j) Y[(size_t)i * r + j] = C[(size_t)j * n + i];
}

// Hermitian eigenproblem of the r x r matrix H (row-major) by cyclic Jacobi rotations;
// on return lam holds eigenvalues in descending order and U (row-major, columns) the
// matching eigenvectors.
static void herm_eig(std::vector<cd> H, int r, std::vector<double> &lam, std::vector<cd> &U) {
    std::vector<cd> E((size_t)r * r, cd(0));
    for (int i = 0; i < r; ++i) E[(size_t)i * r + i] = 1.0;
    auto at = [&](int i, int j) -> cd & { return H[(size_t)i * r + j]; };
    double total = 0;
    for (auto &v : H) total += std::norm(v);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0;
        for (int i = 0; i < r; ++i)
            for (int j = 0; j < r; ++j)
                if (i != j) off += std::norm(at(i, j));
        if (off <= 1e-30 * total) break;
        for (int p = 0; p < r - 1; ++p)
            for (int q = p + 1; q < r; ++q) {
                const cd hpq = at(p, q);
                const double a = std::abs(hpq);
                if (a <= 1e-300) continue;
                const cd ph = hpq / a;                      // e^{i phi}
                const double hpp = at(p, p).real(), hqq = at(q, q).real();
                const double theta = 0.5 * std::atan2(2.0 * a, hqq - hpp);
                const double c = std::cos(theta), s = std::sin(theta);
                // unitary R = [[c, s e^{i phi}], [-s e^{-i phi}, c]] on coordinates p, q;
                // H <- R^H H R zeroes H_pq for tan(2 theta) = 2|H_pq| / (H_qq - H_pp).
                for (int k = 0; k < r; ++k) {
                    const cd xp = at(k, p), xq = at(k, q);
                    at(k, p) = c * xp - s * std::conj(ph) * xq;
                    at(k, q) = s * ph * xp + c * xq;
                }
                for (int k = 0; k < r; ++k) {
                    const cd xp = at(p, k), xq = at(q, k);
                    at(p, k) = c * xp - s * ph * xq;
                    at(q, k) = s * std::conj(ph) * xp + c * xq;
                }
                for (int k = 0; k < r; ++k) {
                    const cd xp = E[(size_t)k * r + p], xq = E[(size_t)k * r + q];
                    E[(size_t)k * r + p] = c * xp - s * std::conj(ph) * xq;
                    E[(size_t)k * r + q] = s * ph * xp + c * xq;
                }
            }
    }
    std::vector<int> order(r);
    for (int i = 0; i < r; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return at(a, a).real() > at(b, b).real(); });
    lam.resize(r);
    U.assign((size_t)r * r, cd(0));
    for (int j = 0; j < r; ++j) {
        lam[j] = at(order[j], order[j]).real();
        for (int i = 0; i < r; ++i) U[(size_t)i * r + j] = E[(size_t)i * r + order[j]];
    }
}

static int rank_rule(const std::vector<double> &s2, double trace, double delta) {
    double cs = 0;
    int K = (int)s2.size();
    for (size_t k = 0; k < s2.size(); ++k) {
        cs += s2[k];
        if (cs >= (1.0 - delta) * trace) {
            K = (int)k + 1;
            break;
        }
    }
    while (K < (int)s2.size() && s2[K] >= s2[K - 1] - 1e-10 * s2[0]) ++K;
    return K;
}

// FP32 device copies of the FP64 host basis: V^T [K][L] and D [Q][K] as complex64, and the
// D rows of the class representatives.
int install_basis(sp_basis *b) {
    const sp_steering *st = b->st;
    const int K = b->K, L = st->L, Q = st->Q;
    std::vector<float> vt((size_t)K * L * 2), dc((size_t)Q * K * 2);
    for (int l = 0; l < L; ++l)
        for (int k = 0; k < K; ++k) {
            vt[((size_t)k * L + l) * 2] = (float)b->V[((size_t)l * K + k) * 2];
            vt[((size_t)k * L + l) * 2 + 1] = (float)b->V[((size_t)l * K + k) * 2 + 1];
        }
    for (size_t i = 0; i < dc.size(); ++i) dc[i] = (float)b->D[i];
    const int nr = (int)st->reps.size();
    std::vector<float> dcr((size_t)nr * K * 2);
    for (int r = 0; r < nr; ++r)
        for (int k = 0; k < 2 * K; ++k) dcr[(size_t)r * K * 2 + k] = dc[(size_t)st->reps[r] * K * 2 + k];
    SP_TRY(b->Dc32r.reserve(dcr.size() * 4));
    SP_CUDA(cudaMemcpy(b->Dc32r.p, dcr.data(), dcr.size() * 4, cudaMemcpyHostToDevice));
    SP_TRY(b->Vc32.reserve(vt.size() * 4));
    SP_TRY(b->Dc32.reserve(dc.size() * 4));
    SP_CUDA(cudaMemcpy(b->Vc32.p, vt.data(), vt.size() * 4, cudaMemcpyHostToDevice));
    SP_CUDA(cudaMemcpy(b->Dc32.p, dc.data(), dc.size() * 4, cudaMemcpyHostToDevice));
    return SP_OK;
}

int reduce_basis(const sp_steering *st, double delta, sp_basis *b) {
    const int Q = st->Q, L = st->L;
    const int nmin = std::min(Q, L);
    DevBuf dW;
    SP_TRY(dW.reserve((size_t)Q * L * 16));
    {
        const long long n = (long long)Q * L;
        w64_kernel<<<(unsigned)((n + 255) / 256), 256>>>(st->tau.as<double>(), Q, st->P, st->B, st->N,
                                                         dW.as<double2>());
        SP_CUDA(cudaGetLastError());
    }
    const double trace = (double)Q * (double)L;
    std::mt19937_64 rng(0x5eed5eedULL);
    std::normal_distribution<double> nd;
    int r = std::min(nmin, 96);
    const int n_power = 4;
    for (int attempt = 0; attempt < 8; ++attempt) {
        DevBuf dA, dB;   // dA: L x r, dB: Q x r
        SP_TRY(dA.reserve((size_t)L * r * 16));
        SP_TRY(dB.reserve((size_t)Q * r * 16));
        std::vector<cd> hA((size_t)L * r), hB((size_t)Q * r);
        for (auto &v : hA) v = cd(nd(rng), nd(rng));
        SP_CUDA(cudaMemcpy(dA.p, hA.data(), hA.size() * 16, cudaMemcpyHostToDevice));
        SP_TRY(zgemm(false, Q, r, L, dW.p, L, dA.p, r, dB.p, r));          // Y = W Omega
        for (int it = 0; it < n_power; ++it) {
            SP_CUDA(cudaMemcpy(hB.data(), dB.p, hB.size() * 16, cudaMemcpyDeviceToHost));
            orthonormalize(hB, Q, r, rng);
            SP_CUDA(cudaMemcpy(dB.p, hB.data(), hB.size() * 16, cudaMemcpyHostToDevice));
            SP_TRY(zgemm(true, L, r, Q, dW.p, L, dB.p, r, dA.p, r));       // H = W^H Y
            SP_CUDA(cudaMemcpy(hA.data(), dA.p, hA.size() * 16, cudaMemcpyDeviceToHost));
            orthonormalize(hA, L, r, rng);
            SP_CUDA(cudaMemcpy(dA.p, hA.data(), hA.size() * 16, cudaMemcpyHostToDevice));
            SP_TRY(zgemm(false, Q, r, L, dW.p, L, dA.p, r, dB.p, r));      // Y = W H
        }
        SP_CUDA(cudaMemcpy(hB.data(), dB.p, hB.size() * 16, cudaMemcpyDeviceToHost));
        orthonormalize(hB, Q, r, rng);
        SP_CUDA(cudaMemcpy(dB.p, hB.data(), hB.size() * 16, cudaMemcpyHostToDevice));
        SP_TRY(zgemm(true, L, r, Q, dW.p, L, dB.p, r, dA.p, r));           // Bh = W^H Y
        DevBuf dG;
        SP_TRY(dG.reserve((size_t)r * r * 16));
        SP_TRY(zgemm(true, r, r, L, dA.p, r, dA.p, r, dG.p, r));           // B B^H = Bh^H Bh
        std::vector<cd> G((size_t)r * r);
        SP_CUDA(cudaMemcpy(G.data(), dG.p, G.size() * 16, cudaMemcpyDeviceToHost));
        for (int i = 0; i < r; ++i)                                        // exact Hermitian
            for (int j = i; j < r; ++j) {
                const cd v = 0.5 * (G[(size_t)i * r + j] + std::conj(G[(size_t)j * r + i]));
                G[(size_t)i * r + j] = v;
                G[(size_t)j * r + i] = std::conj(v);
            }
        std::vector<double> lam;
        std::vector<cd> U;
        herm_eig(G, r, lam, U);
        for (auto &v : lam) v = std::max(v, 0.0);
        const int K = rank_rule(lam, trace, delta);
        const bool enough = (r == nmin) || (K <= r - 24);
        if (!enough) {
            r = std::min(nmin, 2 * r);
            continue;
        }
        // V = Bh U~_K S_K^-1 (L x K)
        SP_CUDA(cudaMemcpy(hA.data(), dA.p, hA.size() * 16, cudaMemcpyDeviceToHost));
        std::vector<cd> V((size_t)L * K);
        for (int l = 0; l < L; ++l)
            for (int k = 0; k < K; ++k) {
                cd acc = 0;
                for (int j = 0; j < r; ++j) acc += hA[(size_t)l * r + j] * U[(size_t)j * r + k];
                V[(size_t)l * K + k] = acc / std::sqrt(lam[k]);
            }
        // D = W V (Q x K) in FP64 on the device
        DevBuf dV, dD;
        SP_TRY(dV.reserve(V.size() * 16));
        SP_TRY(dD.reserve((size_t)Q * K * 16));
        SP_CUDA(cudaMemcpy(dV.p, V.data(), V.size() * 16, cudaMemcpyHostToDevice));
        SP_TRY(zgemm(false, Q, K, L, dW.p, L, dV.p, K, dD.p, K));
        std::vector<cd> D((size_t)Q * K);
        SP_CUDA(cudaMemcpy(D.data(), dD.p, D.size() * 16, cudaMemcpyDeviceToHost));
        b->K = K;
        b->sigma2 = lam;
        b->V.resize(V.size() * 2);
        b->D.resize(D.size() * 2);
        for (size_t i = 0; i < V.size(); ++i) {
            b->V[2 * i] = V[i].real();
            b->V[2 * i + 1] = V[i].imag();
        }
        for (size_t i = 0; i < D.size(); ++i) {
            b->D[2 * i] = D[i].real();
            b->D[2 * i + 1] = D[i].imag();
        }
        SP_TRY(install_basis(b));
        return SP_OK;
    }
    return fail(SP_ENOTIMPL, "svd_reduce: rank did not settle within the block-size limit");
}

}  // namespace sp
