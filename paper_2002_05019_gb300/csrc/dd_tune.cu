// Schedule cache of the autotuner (host only): dd_tune_key,
// dd_tune_cache_lookup, dd_tune_cache_store, declared in include/dd_diag.h,
// and the helpers dd_setup / dd_autotune use.
//
// A factor schedule depends on the problem's front tree and on the GPU.  The
// problem key is a 64-bit FNV-1a hash of the front tree of the symbolic
// analysis (parent, eliminated and update rows of every front), the number of
// duals, the precision and the pivoting mode; the cache key adds the device
// name and its SM count.  The cache is a text file of JSON lines, one per
// tuned problem:
//   {"key": "<16 hex digits>:<device name>:<SMs>", "update_panels": P,
//    "ahead_fronts": A, "reserve_sms": R, "split_sms": S, "factor_ms": T}
// appended by one write per line; a lookup takes the last well-formed line of
// the key and ignores any other line.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/dd.h"
#include "../../include/dd_diag.h"
#include "dd_internal.h"

namespace {

struct Fnv {
  uint64_t h = 1469598103934665603ull;
  void add(int64_t v) {
    for (int b = 0; b < 8; ++b) {
      h ^= (uint64_t)((v >> (8 * b)) & 0xff);
      h *= 1099511628211ull;
    }
  }
};

// the integer after `"name": ` in line, or false
bool json_int(const std::string& line, const char* name, long long* v) {
  const std::string pat = std::string("\"") + name + "\":";
  const size_t p = line.find(pat);
  if (p == std::string::npos) return false;
  return std::sscanf(line.c_str() + p + pat.size(), " %lld", v) == 1;
}

bool json_real(const std::string& line, const char* name, double* v) {
  const std::string pat = std::string("\"") + name + "\":";
  const size_t p = line.find(pat);
  if (p == std::string::npos) return false;
  return std::sscanf(line.c_str() + p + pat.size(), " %lf", v) == 1;
}

// the string value of "key" in line, or false
bool json_key(const std::string& line, std::string* key) {
  const std::string pat = "\"key\": \"";
  const size_t p = line.find(pat);
  if (p == std::string::npos) return false;
  const size_t e = line.find('"', p + pat.size());
  if (e == std::string::npos) return false;
  *key = line.substr(p + pat.size(), e - p - pat.size());
  return true;
}

}  // namespace

uint64_t tune_problem_key(int n_front, const int32_t* parent, const int32_t* ne, const int32_t* nu, int n_dual,
                          int precision, int pivoting) {
  Fnv f;
  f.add(n_front);
  f.add(n_dual);
  f.add(precision);
  f.add(pivoting);
  for (int x = 0; x < n_front; ++x) {
    f.add(parent[x]);
    f.add(ne[x]);
    f.add(nu[x]);
  }
  return f.h;
}

std::string tune_cache_key(uint64_t problem_key, int device) {
  cudaDeviceProp prop{};
  char name[300] = "unknown";
  int sms = 0;
  if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) {
    std::snprintf(name, sizeof(name), "%s", prop.name);
    sms = prop.multiProcessorCount;
  }
  for (char* c = name; *c; ++c)
    if (*c == '"' || *c == ':' || *c == '\\' || *c == '\n') *c = '_';   // keep the key a plain JSON string
  char buf[400];
  std::snprintf(buf, sizeof(buf), "%016llx:%s:%d", (unsigned long long)problem_key, name, sms);
  return buf;
}

extern "C" {

int dd_tune_key(int32_t n_sub, const dd_subdomain* subs, int32_t n_dual, const dd_options* opt, uint64_t* key) {
  if (!key || !opt || n_sub < 1) return DD_ERR_INVALID_ARG;
  // the front tree holds at most 2 n_sub - 1 dense-domain and separator
  // fronts, plus the sparse domains' fronts: grow the arrays until it fits
  for (int64_t cap = 2 * (int64_t)n_sub + 1; cap < (int64_t)1 << 30; cap *= 2) {
    std::vector<int32_t> parent(cap), ne(cap), nu(cap), df(n_dual > 0 ? n_dual : 1);
    int32_t nf = 0;
    const int st = dd_symbolic(n_sub, subs, n_dual, opt, (int32_t)cap, &nf, parent.data(), ne.data(), nu.data(),
                               df.data(), 0, nullptr, nullptr);
    if (st == DD_ERR_INVALID_ARG && nf > cap) continue;
    if (st != DD_OK) return st;
    *key = tune_problem_key(nf, parent.data(), ne.data(), nu.data(), n_dual, opt->precision, opt->pivoting);
    return DD_OK;
  }
  return DD_ERR_INVALID_ARG;
}

int dd_tune_cache_lookup(const char* path, const char* key, dd_schedule* out, int32_t* found) {
  if (!path || !key || !out || !found) return DD_ERR_INVALID_ARG;
  *found = 0;
  std::FILE* fh = std::fopen(path, "r");
  if (!fh) return DD_OK;   // no cache yet
  std::string line;
  char buf[1024];
  while (std::fgets(buf, sizeof(buf), fh)) {
    line.assign(buf);
    std::string k;
    long long p = 0, a = 0, r = 0, sp = 0;
    double t = 0.0;
    if (!json_key(line, &k) || k != key) continue;
    if (!json_int(line, "update_panels", &p) || !json_int(line, "ahead_fronts", &a) ||
        !json_int(line, "reserve_sms", &r) || !json_int(line, "split_sms", &sp) || !json_real(line, "factor_ms", &t))
      continue;
    if ((p != 1 && p != 2 && p != 4) || a < 0 || a > 1024 || r < 0 || r > 64 || sp < 0 || sp > 120) continue;
    out->update_panels = (int32_t)p;
    out->ahead_fronts = (int32_t)a;
    out->reserve_sms = (int32_t)r;
    out->split_sms = (int32_t)sp;
    out->factor_ms = t;
    out->configs_tried = 0;
    *found = 1;
  }
  std::fclose(fh);
  return DD_OK;
}

int dd_tune_cache_store(const char* path, const char* key, const dd_schedule* s) {
  if (!path || !key || !s || std::strchr(key, '"') || std::strchr(key, '\n')) return DD_ERR_INVALID_ARG;
  std::FILE* fh = std::fopen(path, "a");
  if (!fh) return DD_ERR_INVALID_ARG;
  const int n = std::fprintf(fh,
                             "{\"key\": \"%s\", \"update_panels\": %d, \"ahead_fronts\": %d, \"reserve_sms\": %d, "
                             "\"split_sms\": %d, \"factor_ms\": %.6g}\n",
                             key, s->update_panels, s->ahead_fronts, s->reserve_sms, s->split_sms, s->factor_ms);
  const int c = std::fclose(fh);
  return n > 0 && c == 0 ? DD_OK : DD_ERR_INVALID_ARG;
}

}  // extern "C"
