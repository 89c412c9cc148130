// Persistence of the offline results of Algorithm 1 (offline steps 1-3: the geometry that
// defines W, the rank K chosen by Eq. 11, V and D = U S of Eq. 12-13).  The offline phase
// runs once per array and grid; a saved basis lets the online phase start without it.
//
// File layout (little-endian, every field naturally aligned):
//   0   char[8]  magic "SVDPHAT1"
//   8   uint32   version (1)
//   12  uint32   header bytes (80)
//   16  int32    M, Q, N, K, n_sigma, model (0: directions, Eq. 2; 1: source positions, Eq. 1)
//   40  double   fs, c, delta
//   64  uint64   payload bytes (everything after the header, before the checksum)
//   72  uint64   reserved (0)
//   80  double   mic [M][3], dirs (or source positions) [Q][3], sigma2 [n_sigma],
//                V [L][K] complex (re, im), D [Q][K] complex (re, im)
//   end uint64   FNV-1a 64 of every preceding byte
// The device copies (FP32 / FP16 / BF16 operands, direction classes, k-d tree) are rebuilt
// on load from these FP64 values by the same routines sp_svd_reduce uses, so a loaded basis
// gives bit-identical results to the one that was saved.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.h"

namespace sp {
namespace {

constexpr char kMagic[8] = {'S', 'V', 'D', 'P', 'H', 'A', 'T', '1'};
constexpr uint32_t kVersion = 1;
constexpr uint32_t kHeaderBytes = 80;

struct FileHeader {
    char magic[8];
    uint32_t version, header_bytes;
    int32_t M, Q, N, K, n_sigma, model;
    double fs, c, delta;
    uint64_t payload_bytes, reserved1;
};
static_assert(sizeof(FileHeader) == kHeaderBytes, "header layout");

uint64_t fnv1a(const unsigned char *p, size_t n, uint64_t h = 1469598103934665603ULL) {
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ULL;
    }
    return h;
}

// Number of doubles after the header for the given sizes.
size_t payload_doubles(int M, int Q, int N, int K, int n_sigma) {
    const size_t P = (size_t)M * (M - 1) / 2, B = (size_t)N / 2 + 1, L = P * B;
    return 3 * (size_t)M + 3 * (size_t)Q + (size_t)n_sigma + 2 * L * K + 2 * (size_t)Q * K;
}

}  // namespace
}  // namespace sp

using namespace sp;

extern "C" int sp_save_basis(const sp_basis *b, const char *path) {
    SP_CHECK(b && path, SP_EINVAL, "sp_save_basis: null basis or path");
    const sp_steering *st = b->st;
    FileHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, kMagic, 8);
    h.version = kVersion;
    h.header_bytes = kHeaderBytes;
    h.M = st->M;
    h.Q = st->Q;
    h.N = st->N;
    h.K = b->K;
    h.n_sigma = (int32_t)b->sigma2.size();
    h.model = st->nearfield ? 1 : 0;
    h.fs = st->fs;
    h.c = st->c;
    h.delta = b->delta;
    const size_t nd = payload_doubles(h.M, h.Q, h.N, h.K, h.n_sigma);
    h.payload_bytes = nd * 8;
    std::vector<double> body;
    body.reserve(nd);
    body.insert(body.end(), st->mic.begin(), st->mic.end());
    body.insert(body.end(), st->dirs.begin(), st->dirs.end());
    body.insert(body.end(), b->sigma2.begin(), b->sigma2.end());
    body.insert(body.end(), b->V.begin(), b->V.end());
    body.insert(body.end(), b->D.begin(), b->D.end());
    SP_CHECK(body.size() == nd, SP_EINVAL, "sp_save_basis: inconsistent basis sizes");
    uint64_t sum = fnv1a(reinterpret_cast<const unsigned char *>(&h), sizeof h);
    sum = fnv1a(reinterpret_cast<const unsigned char *>(body.data()), nd * 8, sum);
    FILE *f = std::fopen(path, "wb");
    SP_CHECK(f != nullptr, SP_EINVAL, std::string("sp_save_basis: cannot open ") + path);
    bool ok = std::fwrite(&h, sizeof h, 1, f) == 1;
    ok = ok && std::fwrite(body.data(), 8, nd, f) == nd;
    ok = ok && std::fwrite(&sum, 8, 1, f) == 1;
    ok = (std::fclose(f) == 0) && ok;
    SP_CHECK(ok, SP_EINVAL, std::string("sp_save_basis: write failed: ") + path);
    return SP_OK;
}

extern "C" int sp_load_basis(const char *path, int flags, sp_basis **out, int *K_out) {
    SP_CHECK(out, SP_EINVAL, "sp_load_basis: out is NULL");
    *out = nullptr;
    SP_CHECK(path, SP_EINVAL, "sp_load_basis: null path");
    SP_CHECK((flags & ~SP_STEER_MATERIALIZE_W) == 0, SP_EINVAL, "sp_load_basis: bad flags");
    FILE *f = std::fopen(path, "rb");
    SP_CHECK(f != nullptr, SP_EINVAL, std::string("sp_load_basis: cannot open ") + path);
    std::vector<unsigned char> bytes;
    {
        unsigned char buf[1 << 16];
        size_t n;
        while ((n = std::fread(buf, 1, sizeof buf, f)) > 0) bytes.insert(bytes.end(), buf, buf + n);
        std::fclose(f);
    }
    SP_CHECK(bytes.size() >= kHeaderBytes + 8, SP_EINVAL, "sp_load_basis: file too short");
    FileHeader h;
    std::memcpy(&h, bytes.data(), sizeof h);
    SP_CHECK(std::memcmp(h.magic, kMagic, 8) == 0, SP_EINVAL, "sp_load_basis: not a basis file");
    SP_CHECK(h.version == kVersion && h.header_bytes == kHeaderBytes, SP_EINVAL,
             "sp_load_basis: unsupported version");
    SP_CHECK(h.M >= 2 && h.M <= 64 && h.Q >= 1 && h.Q <= (1 << 24) && h.N >= 4 && h.N <= 8192 && h.N % 2 == 0,
             SP_EINVAL, "sp_load_basis: geometry out of range");
    SP_CHECK(h.model == 0 || h.model == 1, SP_EINVAL, "sp_load_basis: unknown steering model");
    const long long L = (long long)h.M * (h.M - 1) / 2 * (h.N / 2 + 1);
    const long long kmax = std::min<long long>(h.Q, L);
    SP_CHECK(h.K >= 1 && h.K <= kmax && h.n_sigma >= h.K && h.n_sigma <= kmax, SP_EINVAL,
             "sp_load_basis: rank out of range");
    const size_t nd = payload_doubles(h.M, h.Q, h.N, h.K, h.n_sigma);
    SP_CHECK(h.payload_bytes == nd * 8 && bytes.size() == kHeaderBytes + nd * 8 + 8, SP_EINVAL,
             "sp_load_basis: file size does not match its header");
    uint64_t sum;
    std::memcpy(&sum, bytes.data() + kHeaderBytes + nd * 8, 8);
    SP_CHECK(fnv1a(bytes.data(), kHeaderBytes + nd * 8) == sum, SP_EINVAL, "sp_load_basis: checksum mismatch");
    std::vector<double> body(nd);
    std::memcpy(body.data(), bytes.data() + kHeaderBytes, nd * 8);
    for (double v : body) SP_CHECK(std::isfinite(v), SP_EINVAL, "sp_load_basis: non-finite value");
    SP_CHECK(h.delta > 0 && h.delta < 1, SP_EINVAL, "sp_load_basis: delta out of range");
    const double *mic = body.data();
    const double *dirs = mic + 3 * h.M;
    const double *sig = dirs + 3 * (size_t)h.Q;
    const double *V = sig + h.n_sigma;
    const double *D = V + 2 * (size_t)L * h.K;

    sp_steering *st = nullptr;
    if (h.model == 1)
        SP_TRY(sp_build_steering_nearfield(mic, h.M, dirs, h.Q, h.fs, h.c, h.N, flags, &st));
    else
        SP_TRY(sp_build_steering(mic, h.M, dirs, h.Q, h.fs, h.c, h.N, flags, &st));
    sp_basis *b = new (std::nothrow) sp_basis();
    if (!b) {
        sp_steering_destroy(st);
        return fail(SP_ENOMEM, "sp_load_basis: host allocation failed");
    }
    b->owned_st = st;
    b->st = st;
    b->K = h.K;
    b->delta = h.delta;
    b->sigma2.assign(sig, sig + h.n_sigma);
    b->V.assign(V, V + 2 * (size_t)L * h.K);
    b->D.assign(D, D + 2 * (size_t)h.Q * h.K);
    int rc = install_basis(b);
    if (rc == SP_OK) rc = build_kdtree(b);
    if (rc == SP_OK) rc = tc_prepare(b);
    if (rc == SP_OK) {
        const cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = fail(SP_ECUDA, std::string("sp_load_basis: ") + cudaGetErrorString(e));
    }
    if (rc != SP_OK) {
        delete b;
        return rc;
    }
    if (K_out) *K_out = b->K;
    *out = b;
    return SP_OK;
}

extern "C" int sp_basis_steering(const sp_basis *b, const sp_steering **out) {
    SP_CHECK(b && out, SP_EINVAL, "sp_basis_steering: null pointer");
    *out = b->st;
    return SP_OK;
}
