// Autotuner of the fused Chebyshev sweep and its cache (aao_autotune, aao_tune_lookup,
// aao_set_tune_cache in include/aao.h).
//
// The fused sweep on the 2D mixed path has three kernels (shared-memory tile, persistent TMA,
// warp strips) and the warp-strip kernel has launch parameters: halo depth S (fused steps per
// launch), segment height H, prefetch distance D and warps per CTA NW.  Which is fastest depends
// on the grid, ell and p (wave quantisation over the SMs, the steps left over after the fused
// launches).  aao_autotune times whole preconditioner applies (CUDA events on the handle's
// stream) for each candidate and keeps the fastest; a JSON file of such results is read back
// by aao_create, keyed by device name, grid, ell and precision.
//
// Cache format (written by paper_2506_03947_gb300/tune.py):
//   {"version": 1, "entries": [{"device": "...", "dim": 2, "n": [n0, n1, n2], "ell": 10,
//     "prec": "mixed", "p": 40, "kernel": "stream", "S": 4, "H": 88, "D": 3, "NW": 8,
//     "us_per_apply": 612.0}, ...]}
// The reader below accepts any JSON and ignores keys it does not know.
#include <algorithm>
#include <cctype>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "aao_ctx.h"

namespace aao {

// ---- a small JSON reader (objects, arrays, strings, numbers, literals) ----------------------

struct JVal {
  enum Kind { kNull, kBool, kNum, kStr, kArr, kObj } kind = kNull;
  double num = 0.0;
  bool b = false;
  std::string str;
  std::vector<JVal> arr;
  std::vector<std::pair<std::string, JVal>> obj;
  const JVal* get(const char* key) const {
    for (const auto& kv : obj)
      if (kv.first == key) return &kv.second;
    return nullptr;
  }
};

struct JParser {
  const char* p;
  const char* end;
  bool ok = true;
  void ws() {
    while (p < end && std::isspace((unsigned char)*p)) ++p;
  }
  bool lit(const char* w) {
    const size_t n = std::strlen(w);
    if ((size_t)(end - p) >= n && std::strncmp(p, w, n) == 0) {
      p += n;
      return true;
    }
    return false;
  }
  std::string string() {
    std::string out;
    ++p;  // opening quote
    while (p < end && *p != '"') {
      if (*p == '\\' && p + 1 < end) {
        ++p;
        const char c = *p;
        if (c == 'n') out += '\n';
        else if (c == 't') out += '\t';
        else if (c == 'u') {
          p += 4;  // non-ASCII escapes are not needed by the cache; keep a placeholder
          out += '?';
        } else out += c;
        ++p;
      } else {
        out += *p++;
      }
    }
    if (p >= end) ok = false;
    else ++p;
    return out;
  }
  JVal value(int depth) {
    JVal v;
    ws();
    if (p >= end || depth > 32) {
      ok = false;
      return v;
    }
    if (*p == '{') {
      v.kind = JVal::kObj;
      ++p;
      ws();
      if (p < end && *p == '}') {
        ++p;
        return v;
      }
      while (ok) {
        ws();
        if (p >= end || *p != '"') {
          ok = false;
          break;
        }
        std::string k = string();
        ws();
        if (p >= end || *p != ':') {
          ok = false;
          break;
        }
        ++p;
        JVal item = value(depth + 1);
        v.obj.emplace_back(std::move(k), std::move(item));
        ws();
        if (p < end && *p == ',') {
          ++p;
          continue;
        }
        if (p < end && *p == '}') {
          ++p;
          break;
        }
        ok = false;
      }
    } else if (*p == '[') {
      v.kind = JVal::kArr;
      ++p;
      ws();
      if (p < end && *p == ']') {
        ++p;
        return v;
      }
      while (ok) {
        v.arr.push_back(value(depth + 1));
        ws();
        if (p < end && *p == ',') {
          ++p;
          continue;
        }
        if (p < end && *p == ']') {
          ++p;
          break;
        }
        ok = false;
      }
    } else if (*p == '"') {
      v.kind = JVal::kStr;
      v.str = string();
    } else if (lit("true")) {
      v.kind = JVal::kBool;
      v.b = true;
    } else if (lit("false")) {
      v.kind = JVal::kBool;
    } else if (lit("null")) {
      v.kind = JVal::kNull;
    } else {
      char* q = nullptr;
      v.kind = JVal::kNum;
      v.num = std::strtod(p, &q);
      if (q == p) ok = false;
      else p = q;
    }
    return v;
  }
};

bool read_file(const char* path, std::string* out) {
  FILE* f = std::fopen(path, "rb");
  if (!f) return false;
  char buf[65536];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) out->append(buf, n);
  std::fclose(f);
  return true;
}

int kind_code(const std::string& k) {
  if (k == "tile") return AAO_STEP_TILE;
  if (k == "tma") return AAO_STEP_TMA;
  if (k == "stream") return AAO_STEP_STREAM;
  return -1;
}

// Find the cache entry for (device, dim, n, ell, prec); an entry with the same p is preferred.
// Returns 1 (found, out = kind, S, H, D, NW), 0 (no entry) or -1 (unreadable or malformed file).
int tune_lookup(const char* path, const char* device, int dim, const int64_t n[3], int ell, int prec, int p,
                int32_t out[5]) {
  std::string text;
  if (!path || !read_file(path, &text)) return -1;
  JParser ps{text.data(), text.data() + text.size()};
  JVal root = ps.value(0);
  if (!ps.ok || root.kind != JVal::kObj) return -1;
  const JVal* ents = root.get("entries");
  if (!ents || ents->kind != JVal::kArr) return -1;
  int best = -1;  // 0: match, 1: match with the same p
  for (const JVal& e : ents->arr) {
    if (e.kind != JVal::kObj) continue;
    const JVal *dv = e.get("device"), *dm = e.get("dim"), *nn = e.get("n"), *el = e.get("ell"), *pr = e.get("prec"),
               *kd = e.get("kernel");
    if (!dv || dv->kind != JVal::kStr || !dm || !nn || nn->kind != JVal::kArr || nn->arr.size() != 3 || !el || !pr ||
        pr->kind != JVal::kStr || !kd || kd->kind != JVal::kStr)
      continue;
    if (device && dv->str != device) continue;
    if ((int)dm->num != dim || (int)el->num != ell) continue;
    if ((pr->str == "mixed" ? AAO_MIXED : AAO_FP64) != prec) continue;
    bool same = true;
    for (int d = 0; d < 3; ++d) same = same && (int64_t)nn->arr[d].num == n[d];
    if (!same) continue;
    const int kc = kind_code(kd->str);
    if (kc < 0) continue;
    const JVal* pp = e.get("p");
    const int score = (pp && (int)pp->num == p) ? 1 : 0;
    if (score <= best) continue;
    best = score;
    out[0] = kc;
    const char* keys[4] = {"S", "H", "D", "NW"};
    for (int k = 0; k < 4; ++k) {
      const JVal* v = e.get(keys[k]);
      out[1 + k] = v ? (int32_t)v->num : 0;
    }
  }
  return best >= 0 ? 1 : 0;
}

std::mutex g_cache_mutex;
std::string g_cache_path;
bool g_cache_set = false;

std::string cache_path() {
  std::lock_guard<std::mutex> lock(g_cache_mutex);
  if (g_cache_set) return g_cache_path;
  const char* env = std::getenv("AAO_TUNE_CACHE");
  return env ? std::string(env) : std::string();
}

// A valid segment height for halo depth S, at least h: H + 2S a multiple of 6 (levels in
// lockstep), or with skew H + 2S + 1 (the skewed schedule of S = 4, one more step per unit).
int round_h(int h, int S, int skew = 0) {
  h = std::max(h, 8);
  while ((h + 2 * S + skew) % 6) ++h;
  return h;
}

}  // namespace aao

namespace aao {

// Configuration (S, D, NW) with the smallest segment height that puts all units of one launch
// into `waves` rounds over the device's warps (units = ell/2 passes x segments x strips of
// 64 - 2S interior columns), at most one segment per strip.
StreamConfig wave_stream_config(const GridDesc& g, int ell, int S, int D, int NW, int waves, int skew) {
  StreamConfig c;
  c.S = S;
  c.D = D;
  c.NW = NW;
  int dev = 0, nsm = 148;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess) {
    cudaGetLastError();
    nsm = 148;
  }
  const int iw = 64 - 2 * S;
  const int nstrip = (g.n0 + iw - 1) / iw;
  const int per_seg = (ell / 2) * nstrip;
  const int segs = std::max(1, waves * nsm * NW / std::max(1, per_seg));
  c.H = round_h((g.n1 + segs - 1) / segs, S, skew);
  if (c.H > round_h(g.n1, S, skew)) c.H = round_h(g.n1, S, skew);
  return c;
}

// The warp-strip configuration used without a cache entry: S = 4 on the skewed schedule, D = 5,
// 8 warps per CTA, one round of units.
StreamConfig default_stream_config(const GridDesc& g, int ell) { return wave_stream_config(g, ell, 4, 5, 8, 1, 1); }

// The two-step final launch: S = 2, D = 3, 16 warps per CTA (the two-step kernel stays within
// 128 registers), one round of units.
StreamConfig default_tail_config(const GridDesc& g, int ell) { return wave_stream_config(g, ell, 2, 3, 16, 1, 0); }

// Apply the cache entry for this handle, if a cache is configured and holds one.
void apply_tune_cache(aao_ctx* h) {
  if (!h->pairs) return;
  const std::string path = cache_path();
  if (path.empty()) return;
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  int32_t out[5] = {0, 0, 0, 0, 0};
  if (tune_lookup(path.c_str(), prop.name, h->dim, h->n, h->ell, h->prec, h->p, out) != 1) return;
  if (out[0] == AAO_STEP_STREAM) {
    StreamConfig c;
    c.S = out[1];
    c.H = out[2];
    c.D = out[3];
    c.NW = out[4];
    if (!stream_config_supported(c)) return;
    h->scfg = c;
  } else if (out[0] == AAO_STEP_TMA && !h->tma) {
    return;
  }
  h->auto_kind = out[0];
  h->tuned = true;
}

}  // namespace aao

extern "C" {

int aao_set_tune_cache(const char* path) {
  std::lock_guard<std::mutex> lock(aao::g_cache_mutex);
  aao::g_cache_set = path != nullptr;
  aao::g_cache_path = path ? path : "";
  return AAO_OK;
}

int aao_tune_lookup(const char* path, const char* device, int dim, const int64_t n[3], int ell, int prec, int p,
                    int32_t out[5]) {
  if (!path || !n || !out) return -AAO_EINVAL;
  const int r = aao::tune_lookup(path, device, dim, n, ell, prec, p, out);
  return r < 0 ? -AAO_EINVAL : r;
}

int aao_get_tuning(aao_handle h, int32_t out[6]) {
  if (!h || !out) return aao::handle_fail(h, AAO_EINVAL, "NULL argument");
  out[0] = aao_get_step_kernel(h);
  out[1] = h->scfg.S;
  out[2] = h->scfg.H;
  out[3] = h->scfg.D;
  out[4] = h->scfg.NW;
  out[5] = h->tuned ? 1 : 0;
  return AAO_OK;
}

int aao_autotune(aao_handle h, int reps, aao_tune_entry* results, int max_results, int* n_results,
                 aao_tune_entry* best) {
  using aao::handle_fail;
  if (!h) return handle_fail(nullptr, AAO_EINVAL, "NULL handle");
  if (!h->pairs || h->pmode != AAO_PRECOND_NC || h->p < 3)
    return handle_fail(h, AAO_EINVAL, "nothing to tune: the fused sweep needs the 2D mixed path with n0 %% 4 == 0, "
                                      "P_NC and inner_its >= 3");
  if (reps < 1 || reps > 1000) return handle_fail(h, AAO_EINVAL, "reps must be in [1, 1000]");
  if (max_results < 0 || (max_results > 0 && !results)) return handle_fail(h, AAO_EINVAL, "bad results buffer");
  int rc = aao::handle_ensure_stage(h);
  if (rc) return rc;
  cudaStream_t s = h->stream;
  cudaError_t e = cudaMemsetAsync(h->stage_a, 0, sizeof(double) * h->L, s);
  if (e != cudaSuccess) return handle_fail(h, AAO_ECUDA, "tuning input: %s", cudaGetErrorString(e));

  int dev = 0, nsm = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();

  // candidates: the tile and TMA kernels, and warp-strip configurations whose segment heights
  // fill one, two or three rounds of units over the device's warps, plus one segment per strip
  // (S = 4 with 6, 8 or 12 warps in lockstep, and with 8 warps on the skewed schedule)
  std::vector<aao_tune_entry> cand;
  auto add = [&](int kind, int S, int H, int D, int NW) {
    aao_tune_entry c{};
    c.kind = kind;
    c.S = S;
    c.H = H;
    c.D = D;
    c.NW = NW;
    c.us_per_apply = -1.0;
    for (const auto& o : cand)
      if (o.kind == kind && o.S == S && o.H == H && o.D == D && o.NW == NW) return;
    cand.push_back(c);
  };
  add(AAO_STEP_TILE, 4, 0, 0, 0);
  if (h->tma) add(AAO_STEP_TMA, 4, 0, 0, 0);
  const int npass = h->ell / 2;
  for (int S : {2, 4}) {
    if (h->p - 2 < S) continue;  // no fused launch would run
    const int nws_s2[] = {8, 12, 16};
    const int nws_s4[] = {6, 8, 12};
    const int* nws = (S == 2) ? nws_s2 : nws_s4;
    const int nnw = (S == 2) ? 3 : 4;
    for (int i = 0; i < nnw; ++i) {
      const int NW = i < 3 ? nws[i] : 8;
      const int skew = i < 3 ? 0 : 1;
      const int nstrip = (h->g.n0 + (64 - 2 * S) - 1) / (64 - 2 * S);
      const int hmax = aao::round_h(h->g.n1, S, skew);
      std::vector<int> hs = {hmax};
      for (int w = 1; w <= 3; ++w) {
        const int segs = w * nsm * NW / std::max(1, npass * nstrip);
        if (segs >= 1) hs.push_back(std::min(hmax, aao::round_h((h->g.n1 + segs - 1) / segs, S, skew)));
      }
      for (int H : hs)
        for (int D : {3, 4, 5}) {  // 5: S = 4 at 8 warps only (stream_config_supported)
          aao::StreamConfig c;
          c.S = S;
          c.H = H;
          c.D = D;
          c.NW = NW;
          if (aao::stream_config_supported(c)) add(AAO_STEP_STREAM, S, H, D, NW);
        }
    }
  }

  const int saved_kind = h->step_kernel, saved_auto = h->auto_kind;
  const aao::StreamConfig saved_cfg = h->scfg, saved_tail = h->tail;
  const bool saved_prof = h->prof;
  h->prof = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // time candidates [i0, cand.size()): whole applies with the candidate set on the handle
  // (a sweep candidate, or with tail = 1 a two-step final launch under the best sweep)
  auto run = [&](size_t i0, int& best_i) {
    for (size_t i = i0; i < cand.size() && e == cudaSuccess && rc == AAO_OK; ++i) {
      aao_tune_entry& c = cand[i];
      aao::StreamConfig& dst = c.tail ? h->tail : h->scfg;
      if (!c.tail) h->step_kernel = c.kind;
      if (c.kind == AAO_STEP_STREAM) {
        dst.S = c.S;
        dst.H = c.H;
        dst.D = c.D;
        dst.NW = c.NW;
      }
      rc = aao::handle_precond(h, h->stage_a, nullptr, h->stage_b);  // warm-up
      for (int r = 0; r < reps && rc == AAO_OK; ++r) {
        if (r == 0 && (e = cudaEventRecord(e0, s)) != cudaSuccess) break;
        rc = aao::handle_precond(h, h->stage_a, nullptr, h->stage_b);
      }
      if (rc == AAO_OK && e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (rc == AAO_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (rc == AAO_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (rc == AAO_OK) rc = aao::handle_check_tma(h);
      if (rc == AAO_OK && e == cudaSuccess) {
        c.us_per_apply = 1e3 * ms / reps;
        if (best_i < 0 || c.us_per_apply < cand[best_i].us_per_apply) best_i = (int)i;
      }
    }
  };
  int best_i = -1, tail_i = -1;
  run(0, best_i);
  // the two-step final launch, when the best sweep has S = 4 and the remaining step count
  // (after at most one single step) is 2 mod 4: NW in {8, 12, 16}, D in {3, 4}, one to three
  // rounds of units
  int R = h->p - 2;
  if (R % 2) --R;
  if (rc == AAO_OK && e == cudaSuccess && best_i >= 0 && cand[best_i].kind == AAO_STEP_STREAM &&
      cand[best_i].S == 4 && R >= 2 && R % 4 == 2) {
    const aao_tune_entry b = cand[best_i];
    h->step_kernel = AAO_STEP_STREAM;
    h->scfg.S = b.S;
    h->scfg.H = b.H;
    h->scfg.D = b.D;
    h->scfg.NW = b.NW;
    const size_t i0 = cand.size();
    for (int NW : {8, 12, 16})
      for (int D : {3, 4})
        for (int w = 1; w <= 3; ++w) {
          const aao::StreamConfig c = aao::wave_stream_config(h->g, h->ell, 2, D, NW, w, 0);
          bool dup = false;
          for (size_t i = i0; i < cand.size(); ++i)
            dup = dup || (cand[i].H == c.H && cand[i].D == D && cand[i].NW == NW);
          if (dup || !aao::stream_config_supported(c)) continue;
          aao_tune_entry t{};
          t.kind = AAO_STEP_STREAM;
          t.S = 2;
          t.H = c.H;
          t.D = D;
          t.NW = NW;
          t.tail = 1;
          t.us_per_apply = -1.0;
          cand.push_back(t);
        }
    run(i0, tail_i);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  h->prof = saved_prof;
  h->step_kernel = saved_kind;
  h->auto_kind = saved_auto;
  h->scfg = saved_cfg;
  h->tail = saved_tail;
  aao::handle_reset_graphs(h);
  if (rc) return rc;
  if (e != cudaSuccess) return handle_fail(h, AAO_ECUDA, "tuning: %s", cudaGetErrorString(e));
  if (best_i < 0) return handle_fail(h, AAO_ECUDA, "tuning: no candidate ran");
  // the fastest candidate becomes the handle's default kernel, the fastest tail its final launch
  const aao_tune_entry& b = cand[best_i];
  h->step_kernel = AAO_STEP_AUTO;
  h->auto_kind = b.kind;
  if (b.kind == AAO_STEP_STREAM) {
    h->scfg.S = b.S;
    h->scfg.H = b.H;
    h->scfg.D = b.D;
    h->scfg.NW = b.NW;
  }
  if (tail_i >= 0) {
    const aao_tune_entry& t = cand[tail_i];
    h->tail.S = 2;
    h->tail.H = t.H;
    h->tail.D = t.D;
    h->tail.NW = t.NW;
  }
  h->tuned = true;
  if (best) *best = b;
  if (n_results) *n_results = (int)cand.size();
  for (int i = 0; i < std::min<int>(max_results, (int)cand.size()); ++i) results[i] = cand[i];
  return AAO_OK;
}

}  // extern "C"
