// Offline step 1 of Algorithm 1: the TDOA table (Eq. 2 in the far field, Eq. 1 for sources
// at given positions) and the steering matrix W (Eq. 4, stacked as Eq. 8).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>

#include "common.h"

namespace sp {

// ||s - r|| in the fixed order sqrt((ex*ex + ey*ey) + ez*ez), e = s - r.
__device__ __forceinline__ double dist_rn(double sx, double sy, double sz, const double *r) {
    const double ex = __dsub_rn(sx, r[0]), ey = __dsub_rn(sy, r[1]), ez = __dsub_rn(sz, r[2]);
    return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)));
}

// Far field (Eq. 2): tau[q][p] = fs/c * (r_j - r_i) . s_q / ||s_q||, one thread per (q, p).
// Fixed order, every operation correctly rounded and never contracted into an FMA:
//   n = sqrt((sx*sx + sy*sy) + sz*sz), u = s / n,
//   tau = (fs / c) * ((dx*ux + dy*uy) + dz*uz), d = r_j - r_i.
// Near field (Eq. 1, s_q a source position): tau = (fs / c) * (||s_q - r_i|| - ||s_q - r_j||)
// with each norm in the order of dist_rn.  The same order on any IEEE-754 machine gives the
// same bits.  unit[q] = s_q / ||s_q|| in both cases.
__global__ void tau_kernel(const double *__restrict__ mic, const double *__restrict__ dirs,
                           const int *__restrict__ pi, const int *__restrict__ pj, int Q, int P,
                           double fs, double c, int nearfield, double *__restrict__ tau, double *__restrict__ unit) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)Q * P) return;
    const int q = (int)(idx / P), p = (int)(idx % P);
    const double sx = dirs[3 * q], sy = dirs[3 * q + 1], sz = dirs[3 * q + 2];
    const double n = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(sx, sx), __dmul_rn(sy, sy)),
                                          __dmul_rn(sz, sz)));
    const double ux = __ddiv_rn(sx, n), uy = __ddiv_rn(sy, n), uz = __ddiv_rn(sz, n);
    const int i = pi[p], j = pj[p];
    const double g = __ddiv_rn(fs, c);
    if (nearfield) {
        tau[idx] = __dmul_rn(g, __dsub_rn(dist_rn(sx, sy, sz, mic + 3 * i), dist_rn(sx, sy, sz, mic + 3 * j)));
    } else {
        const double dx = __dsub_rn(mic[3 * j], mic[3 * i]);
        const double dy = __dsub_rn(mic[3 * j + 1], mic[3 * i + 1]);
        const double dz = __dsub_rn(mic[3 * j + 2], mic[3 * i + 2]);
        const double dot = __dadd_rn(__dadd_rn(__dmul_rn(dx, ux), __dmul_rn(dy, uy)), __dmul_rn(dz, uz));
        tau[idx] = __dmul_rn(g, dot);
    }
    if (p == 0) {
        unit[3 * q] = ux;
        unit[3 * q + 1] = uy;
        unit[3 * q + 2] = uz;
    }
}

// W[q][p*B + k] = exp(2 pi i k tau[q][p] / N)  (Eq. 4, Eq. 8), complex64.
// The phase k*tau/N (in turns) is reduced to [-1/2, 1/2] in FP64 before sincospi.
__global__ void w_kernel(const double *__restrict__ tau, int Q, int P, int B, int N,
                         float2 *__restrict__ W) {
    const long long L = (long long)P * B;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)Q * L) return;
    const long long q = idx / L;
    const int l = (int)(idx % L);
    const int p = l / B, k = l % B;
    const double turns = (double)k * tau[q * P + p] / (double)N;
    const double r = turns - rint(turns);
    double s, co;
    sincospi(2.0 * r, &s, &co);
    W[idx] = make_float2((float)co, (float)s);
}

// Per direction q and microphone m, for online step 4: d_m / N in turns per bin, split as
// float hi + lo, and the phasor exp(-2 pi i 64 d_m / N) of a 64-bin step, where
// tau_{q,i,j} = d_j - d_i: d_m = fs/c r_m . u_q in the far field (Eq. 2) and
// d_m = -fs/c ||s_q - r_m|| in the near field (Eq. 1), in FP64.  Computed once here so that
// the step-4 kernel does no FP64 work per frame.
__global__ void step4_table_kernel(const double *__restrict__ mic, const double *__restrict__ unit,
                                   const double *__restrict__ pos, int nearfield, int Q, int M, double g,
                                   double inv_n, float4 *__restrict__ tab) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)Q * M) return;
    const int q = (int)(idx / M), m = (int)(idx % M);
    const double d =
        nearfield ? -g * dist_rn(pos[3 * q], pos[3 * q + 1], pos[3 * q + 2], mic + 3 * m)
                  : g * ((mic[3 * m] * unit[3 * q] + mic[3 * m + 1] * unit[3 * q + 1]) + mic[3 * m + 2] * unit[3 * q + 2]);
    const double e = d * inv_n;
    const float hi = (float)e;
    const float lo = (float)(e - (double)hi);
    const float p1 = 64.f * hi;
    const float r1 = (p1 - rintf(p1)) + 64.f * lo;
    float ss, sc;
    sincospif(-2.f * r1, &ss, &sc);
    tab[idx] = make_float4(hi, lo, sc, ss);
}

int launch_tau(const sp_steering *st, cudaStream_t s) {
    sp_steering *m = const_cast<sp_steering *>(st);
    SP_TRY(m->tau.reserve((size_t)st->Q * st->P * 8));
    SP_TRY(m->d_mic.reserve((size_t)st->M * 3 * 8));
    SP_TRY(m->d_dirs.reserve((size_t)st->Q * 3 * 8));
    DevBuf d_dirs_in, d_pairs;
    SP_TRY(d_dirs_in.reserve((size_t)st->Q * 3 * 8));
    SP_TRY(d_pairs.reserve((size_t)st->P * 2 * 4));
    SP_CUDA(cudaMemcpy(m->d_mic.p, st->mic.data(), st->mic.size() * 8, cudaMemcpyHostToDevice));
    SP_CUDA(cudaMemcpy(d_dirs_in.p, st->dirs.data(), st->dirs.size() * 8, cudaMemcpyHostToDevice));
    SP_CUDA(cudaMemcpy(d_pairs.p, st->pair_i.data(), st->P * 4, cudaMemcpyHostToDevice));
    SP_CUDA(cudaMemcpy(d_pairs.as<int>() + st->P, st->pair_j.data(), st->P * 4, cudaMemcpyHostToDevice));
    const long long n = (long long)st->Q * st->P;
    tau_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
        m->d_mic.as<double>(), d_dirs_in.as<double>(), d_pairs.as<int>(), d_pairs.as<int>() + st->P,
        st->Q, st->P, st->fs, st->c, st->nearfield ? 1 : 0, m->tau.as<double>(), m->d_dirs.as<double>());
    SP_CUDA(cudaGetLastError());
    {
        const long long nm = (long long)st->Q * st->M;
        SP_TRY(m->step4_tab.reserve((size_t)nm * 16));
        step4_table_kernel<<<(unsigned)((nm + 255) / 256), 256, 0, s>>>(
            m->d_mic.as<double>(), m->d_dirs.as<double>(), d_dirs_in.as<double>(), st->nearfield ? 1 : 0, st->Q,
            st->M, st->fs / st->c, 1.0 / (double)st->N, m->step4_tab.as<float4>());
        SP_CUDA(cudaGetLastError());
    }
    SP_CUDA(cudaStreamSynchronize(s));  // the temporaries are freed on return
    return SP_OK;
}

// Equivalence classes of directions: q ~ q' when max_p |tau[q][p] - tau[q'][p]| <= 1e-9
// samples (a line array cannot tell directions on a cone apart, a planar array mirror
// images).  Sort by the first pair's TDOA, compare rows inside the 1e-9 window, join
// classes with union-find; each class is represented by its lowest index.
int build_classes(sp_steering *st) {
    const int Q = st->Q, P = st->P;
    const double tol = 1e-9;
    const double *tau = st->tau_host.data();
    std::vector<int> order(Q), parent(Q);
    std::iota(order.begin(), order.end(), 0);
    std::iota(parent.begin(), parent.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return tau[(size_t)a * P] < tau[(size_t)b * P]; });
    auto find = [&](int x) {
        while (parent[x] != x) {
            parent[x] = parent[parent[x]];
            x = parent[x];
        }
        return x;
    };
    for (int a = 0; a < Q; ++a) {
        const int qa = order[a];
        for (int b = a + 1; b < Q; ++b) {
            const int qb = order[b];
            if (tau[(size_t)qb * P] - tau[(size_t)qa * P] > tol) break;
            bool same = true;
            for (int p = 0; p < P && same; ++p)
                same = std::fabs(tau[(size_t)qa * P + p] - tau[(size_t)qb * P + p]) <= tol;
            if (same) {
                const int ra = find(qa), rb = find(qb);
                if (ra != rb) parent[std::max(ra, rb)] = std::min(ra, rb);
            }
        }
    }
    st->rep_of.resize(Q);
    st->reps.clear();
    for (int q = 0; q < Q; ++q) {
        st->rep_of[q] = find(q);
        if (st->rep_of[q] == q) st->reps.push_back(q);
    }
    SP_TRY(st->d_reps.reserve(st->reps.size() * 4));
    SP_CUDA(cudaMemcpy(st->d_reps.p, st->reps.data(), st->reps.size() * 4, cudaMemcpyHostToDevice));
    return SP_OK;
}

int launch_w(const sp_steering *st, cudaStream_t s) {
    sp_steering *m = const_cast<sp_steering *>(st);
    const long long n = (long long)st->Q * st->L;
    SP_TRY(m->W.reserve((size_t)n * 8));
    w_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(st->tau.as<double>(), st->Q, st->P, st->B,
                                                         st->N, m->W.as<float2>());
    SP_CUDA(cudaGetLastError());
    m->has_w = true;
    return SP_OK;
}

}  // namespace sp
