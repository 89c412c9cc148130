// Autotune cache of batch plans: a JSON file that maps a batch signature (device, mode,
// precision and every stream's shape) to the launch shape the autotuner measured fastest,
// so that a later plan for the same batch skips the measurement.
//
//   {
//     "format": "svdphat-tune-cache",
//     "version": 1,
//     "plans": {
//       "<key>": {"branches": 32, "tiles_per_cta": 1, "proj_variant": 0, "grouped": 1, "ms": 8.17},
//       ...
//     }
//   }
//
// Keys are printable ASCII without '"' or '\'.  The file is rewritten whole (entries sorted
// by key) through a temporary file and a rename, so a reader never sees half a file; a file
// that does not parse is never overwritten.  Host code only.
#include <unistd.h>

#include <cerrno>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "common.h"

namespace sp {
namespace {

std::mutex g_mu;
std::string g_path;   // empty: no cache

bool valid_key(const std::string &k) {
    if (k.empty() || k.size() > 512) return false;
    for (char c : k)
        if (c < 0x20 || c > 0x7e || c == '"' || c == '\\') return false;
    return true;
}

void skip_ws(const std::string &s, size_t &i) {
    while (i < s.size() && (s[i] == ' ' || s[i] == '\t' || s[i] == '\n' || s[i] == '\r')) ++i;
}

// value of "name": <number> inside obj; false if absent or not a number
bool field(const std::string &obj, const char *name, double *v) {
    const std::string pat = std::string("\"") + name + "\"";
    size_t i = obj.find(pat);
    if (i == std::string::npos) return false;
    i += pat.size();
    skip_ws(obj, i);
    if (i >= obj.size() || obj[i] != ':') return false;
    ++i;
    skip_ws(obj, i);
    const char *b = obj.c_str() + i;
    char *e = nullptr;
    errno = 0;
    const double x = std::strtod(b, &e);
    if (e == b || errno != 0) return false;
    *v = x;
    return true;
}

// Parses the whole file into entries.  Returns SP_OK (a missing file is an empty cache) or
// SP_EINVAL for a file that does not parse.
int load(const std::string &path, std::map<std::string, TunedShape> *out) {
    out->clear();
    FILE *f = std::fopen(path.c_str(), "rb");
    if (!f) return errno == ENOENT ? SP_OK : fail(SP_EINVAL, "tune cache: cannot open " + path);
    std::string s;
    char buf[4096];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) s.append(buf, n);
    std::fclose(f);
    const auto bad = [&]() { return fail(SP_EINVAL, "tune cache: " + path + " is not a tune-cache file"); };
    if (s.find("\"svdphat-tune-cache\"") == std::string::npos) return bad();
    size_t i = s.find("\"plans\"");
    if (i == std::string::npos) return bad();
    i += 7;
    skip_ws(s, i);
    if (i >= s.size() || s[i] != ':') return bad();
    ++i;
    skip_ws(s, i);
    if (i >= s.size() || s[i] != '{') return bad();
    ++i;
    while (true) {
        skip_ws(s, i);
        if (i >= s.size()) return bad();
        if (s[i] == '}') break;
        if (s[i] != '"') return bad();
        const size_t k1 = s.find('"', i + 1);
        if (k1 == std::string::npos) return bad();
        const std::string key = s.substr(i + 1, k1 - i - 1);
        i = k1 + 1;
        skip_ws(s, i);
        if (i >= s.size() || s[i] != ':') return bad();
        ++i;
        skip_ws(s, i);
        if (i >= s.size() || s[i] != '{') return bad();
        const size_t o1 = s.find('}', i);
        if (o1 == std::string::npos) return bad();
        const std::string obj = s.substr(i, o1 - i + 1);
        i = o1 + 1;
        double br, tpc, pv, ms, gr = 0.0;
        if (!valid_key(key) || !field(obj, "branches", &br) || !field(obj, "tiles_per_cta", &tpc) ||
            !field(obj, "proj_variant", &pv) || !field(obj, "ms", &ms))
            return bad();
        field(obj, "grouped", &gr);   // optional (0 when absent)
        (*out)[key] = TunedShape{(int)br, (int)tpc, (int)pv, (float)ms, (int)gr};
        skip_ws(s, i);
        if (i < s.size() && s[i] == ',') ++i;
    }
    return SP_OK;
}

int save(const std::string &path, const std::map<std::string, TunedShape> &m) {
    const std::string tmp = path + ".tmp." + std::to_string((long)getpid());
    FILE *f = std::fopen(tmp.c_str(), "wb");
    if (!f) return fail(SP_EINVAL, "tune cache: cannot write " + tmp);
    std::fprintf(f, "{\n  \"format\": \"svdphat-tune-cache\",\n  \"version\": 1,\n  \"plans\": {");
    bool first = true;
    for (const auto &kv : m) {
        std::fprintf(f,
                     "%s\n    \"%s\": {\"branches\": %d, \"tiles_per_cta\": %d, \"proj_variant\": %d, "
                     "\"grouped\": %d, \"ms\": %.6g}",
                     first ? "" : ",", kv.first.c_str(), kv.second.branches, kv.second.tiles_per_cta,
                     kv.second.proj_variant, kv.second.grouped, (double)kv.second.ms);
        first = false;
    }
    std::fprintf(f, "\n  }\n}\n");
    const bool ok = std::fflush(f) == 0;
    std::fclose(f);
    if (!ok || std::rename(tmp.c_str(), path.c_str()) != 0) {
        std::remove(tmp.c_str());
        return fail(SP_EINVAL, "tune cache: cannot replace " + path);
    }
    return SP_OK;
}

}  // namespace

bool tune_cache_enabled() {
    std::lock_guard<std::mutex> lk(g_mu);
    return !g_path.empty();
}

int tune_cache_get(const std::string &key, TunedShape *out, bool *found) {
    *found = false;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_path.empty()) return SP_OK;
    SP_CHECK(valid_key(key), SP_EINVAL, "tune cache: bad key");
    std::map<std::string, TunedShape> m;
    SP_TRY(load(g_path, &m));
    const auto it = m.find(key);
    if (it != m.end()) {
        *out = it->second;
        *found = true;
    }
    return SP_OK;
}

int tune_cache_put(const std::string &key, const TunedShape &v) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_path.empty()) return SP_OK;
    SP_CHECK(valid_key(key), SP_EINVAL, "tune cache: bad key");
    SP_CHECK(v.branches >= 1 && (v.tiles_per_cta == 1 || v.tiles_per_cta == 2 || v.tiles_per_cta == 4) &&
                 (v.proj_variant == 0 || v.proj_variant == 1) && (v.grouped == 0 || v.grouped == 1) && v.ms >= 0.f,
             SP_EINVAL, "tune cache: bad shape");
    std::map<std::string, TunedShape> m;
    SP_TRY(load(g_path, &m));   // a file that does not parse is left alone
    m[key] = v;
    return save(g_path, m);
}

}  // namespace sp

using namespace sp;

extern "C" {

int sp_set_tune_cache(const char *path) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_path = path ? std::string(path) : std::string();
    return SP_OK;
}

int sp_tune_cache_get(const char *key, int *branches, int *tiles_per_cta, int *proj_variant, float *ms, int *grouped,
                      int *found) {
    SP_CHECK(key && found, SP_EINVAL, "sp_tune_cache_get: null pointer");
    TunedShape v{0, 0, 0, 0.f, 0};
    bool f = false;
    SP_TRY(tune_cache_get(key, &v, &f));
    *found = f ? 1 : 0;
    if (f) {
        if (branches) *branches = v.branches;
        if (tiles_per_cta) *tiles_per_cta = v.tiles_per_cta;
        if (proj_variant) *proj_variant = v.proj_variant;
        if (ms) *ms = v.ms;
        if (grouped) *grouped = v.grouped;
    }
    return SP_OK;
}

int sp_tune_cache_put(const char *key, int branches, int tiles_per_cta, int proj_variant, float ms, int grouped) {
    SP_CHECK(key, SP_EINVAL, "sp_tune_cache_put: null key");
    return tune_cache_put(key, TunedShape{branches, tiles_per_cta, proj_variant, ms, grouped});
}

}  // extern "C"
