// Autotuner of the mixed path's fused-kernel launch (the GPU analogue of the paper's block-size
// study, Section 5: the loop tiles are tuned empirically on the target machine).
//
// Candidates: the one-CTA shape (1 x 1 cluster, 16 epilogue warps) for every p; for p = 4 also
// the one-CTA shape with 8 epilogue warps and the CTA pair (cta_group::2); each with 4, 8, 16,
// 32 or 64 SNP tiles per traversal group.  Every candidate solves the same sample of the grid (the first
// SNPs and traits of the problem, device output) once untimed and twice timed with CUDA events;
// the fastest wins, but the default shape is kept when it is within 2 % of it (a plateau, not a
// noisy optimum).  The choice is stored in the context and, when opts.tune_cache names a file,
// in a JSON object keyed by (n, p, mode, t rounded down to a power of two) that gwas_setup
// reads back.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "fused.cuh"
#include "gwas_internal.cuh"

namespace {

std::string tune_key(const gwas_ctx* c, int t) {
  int lg = 0;
  while (lg < 30 && (1 << (lg + 1)) <= t) ++lg;
  char buf[128];
  snprintf(buf, sizeof buf, "n=%d,p=%d,mode=%s,t=2^%d", c->n, c->p, c->precision == GWAS_MIXED ? "mixed" : "fp64", lg);
  return buf;
}

void skip_ws(const std::string& s, size_t& i) {
  while (i < s.size() && (s[i] == ' ' || s[i] == '\n' || s[i] == '\r' || s[i] == '\t')) ++i;
}

// The cache file: one JSON object whose values are flat objects of integers and numbers, as
// written by write_cache.  Returns key -> the text of its object ("{...}"); an unreadable or
// malformed file reads as empty.
std::map<std::string, std::string> read_cache(const std::string& path) {
  std::map<std::string, std::string> out;
  std::ifstream f(path);
  if (!f) return out;
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string s = ss.str();
  size_t i = 0;
  skip_ws(s, i);
  if (i >= s.size() || s[i] != '{') return {};
  ++i;
  for (;;) {
    skip_ws(s, i);
    if (i < s.size() && s[i] == '}') break;
    if (i >= s.size() || s[i] != '"') return {};
    const size_t k0 = ++i;
    while (i < s.size() && s[i] != '"') ++i;
    if (i >= s.size()) return {};
    const std::string key = s.substr(k0, i - k0);
    ++i;
    skip_ws(s, i);
    if (i >= s.size() || s[i] != ':') return {};
    ++i;
    skip_ws(s, i);
    if (i >= s.size() || s[i] != '{') return {};
    const size_t o0 = i;
    while (i < s.size() && s[i] != '}') ++i;
    if (i >= s.size()) return {};
    out[key] = s.substr(o0, i - o0 + 1);
    ++i;
    skip_ws(s, i);
    if (i < s.size() && s[i] == ',') {
      ++i;
      continue;
    }
    if (i < s.size() && s[i] == '}') break;
    return {};
  }
  return out;
}

bool get_int(const std::string& obj, const char* name, int* v) {
  const std::string pat = std::string("\"") + name + "\"";
  size_t i = obj.find(pat);
  if (i == std::string::npos) return false;
  i = obj.find(':', i + pat.size());
  if (i == std::string::npos) return false;
  char* end = nullptr;
  const long x = strtol(obj.c_str() + i + 1, &end, 10);
  if (end == obj.c_str() + i + 1) return false;
  *v = (int)x;
  return true;
}

bool write_cache(const std::string& path, const std::map<std::string, std::string>& m) {
  const std::string tmp = path + ".tmp";
  {
    std::ofstream f(tmp);
    if (!f) return false;
    f << "{\n";
    size_t k = 0;
    for (const auto& e : m) f << "  \"" << e.first << "\": " << e.second << (++k < m.size() ? ",\n" : "\n");
    f << "}\n";
    if (!f) return false;
  }
  return std::rename(tmp.c_str(), path.c_str()) == 0;
}

bool same(const gwas_ctx::FusedTune& a, const gwas_ctx::FusedTune& b) {
  return a.cs == b.cs && a.ct == b.ct && a.epw == b.epw && a.pair == b.pair && a.group == b.group;
}

}  // namespace

void tune_apply_cache(gwas_ctx* c) {
  if (c->tune_cache.empty()) return;
  const auto m = read_cache(c->tune_cache);
  const auto it = m.find(tune_key(c, c->t));
  if (it == m.end()) return;
  gwas_ctx::FusedTune t;
  if (!get_int(it->second, "cs", &t.cs) || !get_int(it->second, "ct", &t.ct) || !get_int(it->second, "epw", &t.epw) ||
      !get_int(it->second, "pair", &t.pair) || !get_int(it->second, "group", &t.group))
    return;
  if (t.group >= 1 && fused_shape_supported(c->pm1, t.cs, t.ct, t.epw, t.pair)) c->tune = t;
}

extern "C" int gwas_autotune(gwas_ctx* c, const double* Y, int t_sample, int64_t m_sample, double* best_ms) {
  if (!c) return GWAS_ERR_ARG;
  if (!Y) return ctx_fail(c, GWAS_ERR_ARG, "NULL Y");
  if (c->precision != GWAS_MIXED) return ctx_fail(c, GWAS_ERR_UNSUPPORTED, "only the mixed path has launch shapes to tune");
  if (c->m == 0) return ctx_fail(c, GWAS_ERR_STATE, "gwas_autotune before gwas_load_snps");
  if (c->serve) return ctx_fail(c, GWAS_ERR_STATE, "gwas_autotune while the serving loop runs");
  DeviceGuard guard(c->device);
  const int ts = std::min(c->t, t_sample > 0 ? t_sample : 1024);
  const int64_t ms = std::min(c->m, m_sample > 0 ? m_sample : (int64_t)1 << 17);
  float* out = nullptr;
  int rc = ctx_alloc(c, sizeof(float) * 2 * (size_t)ts * (size_t)ms, (void**)&out);
  if (rc) return rc;
  std::vector<gwas_ctx::FusedTune> cand;
  const int shapes[3][4] = {{1, 1, 16, 0}, {1, 1, 8, 0}, {2, 1, 16, 1}};
  for (const auto& sh : shapes)
    if (fused_shape_supported(c->pm1, sh[0], sh[1], sh[2], sh[3]))
      for (int g : {16, 4, 8, 32, 64}) cand.push_back({sh[0], sh[1], sh[2], sh[3], g});
  const gwas_ctx::FusedTune saved = c->tune;
  const int saved_t = c->t;
  const bool saved_prof = c->profile;
  c->t = ts;
  c->profile = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<float> times(cand.size(), 1e30f);
  for (size_t k = 0; k < cand.size() && rc == GWAS_OK; ++k) {
    c->tune = cand[k];
    for (int rep = 0; rep < 3 && rc == GWAS_OK; ++rep) {
      cudaEventRecord(e0, c->stream);
      int r = gwas_solve(c, Y, 0, ms, out);
      cudaEventRecord(e1, c->stream);
      if (r != GWAS_OK && r != GWAS_ERR_SINGULAR_PAIRS) {
        rc = r;
        break;
      }
      float t_ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t_ms, e0, e1) != cudaSuccess) {
        cudaGetLastError();
        rc = ctx_fail(c, GWAS_ERR_CUDA, "autotune timing");
        break;
      }
      if (rep > 0) times[k] = std::min(times[k], t_ms);  // the first run is the warm-up
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->t = saved_t;
  c->profile = saved_prof;
  ctx_free(c, out);
  if (rc != GWAS_OK) {
    c->tune = saved;
    return rc;
  }
  size_t best = 0;
  for (size_t k = 1; k < cand.size(); ++k)
    if (times[k] < times[best]) best = k;
  // a plateau, not a noisy optimum: keep the default unless the winner is more than 2 % faster
  const gwas_ctx::FusedTune dflt{};
  for (size_t k = 0; k < cand.size(); ++k)
    if (same(cand[k], dflt) && times[k] <= 1.02f * times[best]) best = k;
  c->tune = cand[best];
  if (best_ms) *best_ms = times[best];
  if (!c->tune_cache.empty()) {
    auto m = read_cache(c->tune_cache);
    char obj[256];
    snprintf(obj, sizeof obj, "{\"cs\": %d, \"ct\": %d, \"epw\": %d, \"pair\": %d, \"group\": %d, \"ms\": %.4f}",
             c->tune.cs, c->tune.ct, c->tune.epw, c->tune.pair, c->tune.group, (double)times[best]);
    m[tune_key(c, c->t)] = obj;
    if (!write_cache(c->tune_cache, m)) return ctx_fail(c, GWAS_ERR_ARG, "cannot write the tune cache " + c->tune_cache);
  }
  return GWAS_OK;
}

extern "C" int gwas_tune_shape(const gwas_ctx* c, int* shape) {
  if (!c || !shape) return GWAS_ERR_ARG;
  shape[0] = c->tune.cs;
  shape[1] = c->tune.ct;
  shape[2] = c->tune.epw;
  shape[3] = c->tune.pair;
  shape[4] = c->tune.group;
  return GWAS_OK;
}
