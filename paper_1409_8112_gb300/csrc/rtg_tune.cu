// Autotuner of the radix sort: digit width (8, 9, 10 or 11 bits per pass), tile size (256 x 8, 12
// or 16 keys) and pass strategy (look-back, reduce-then-scan, or all passes in one cooperative
// launch when every tile fits on the GPU at once).  On the second build of a
// shape it times every variant five times on the build's own keys, each as a replayed CUDA
// graph (the form the build runs it in, so that variants of several launches are not charged
// the gaps of direct launches), and keeps the lowest median, per (sorted elements, key bits),
// in the context and, when RTG_TUNE_CACHE names a file, in a JSON cache shared by later
// contexts and processes.  The same build also times the in-cell enumeration over spans per
// warp {1, 2, 4} and the dense-cell threshold {64, 128, 256} on the sorted keys and keeps the
// fastest (in the context).
// The sort is stable in every variant, so the choice never changes a result.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "rtg_host.h"

namespace rtghost {

namespace {

constexpr int kTuneReps = 5;  // trials per candidate; the median decides (noise-robust)

double median_of(std::vector<double> v) {
  if (v.empty()) return 1e30;
  std::sort(v.begin(), v.end());
  return v[v.size() / 2];
}

// Every compiled variant; the single-launch strategy only where all of its tiles can be
// resident at once (num_sms = 0: every variant, for sizing the scratch).
std::vector<rtg::SortConfig> candidates(long long N = 0, int num_sms = 0, bool key64 = false) {
  std::vector<rtg::SortConfig> v;
  for (int bits : rtg::kSortBitsChoices)
    for (int items : rtg::kSortItemsChoices)
      for (int mode : {rtg::kSortLookback, rtg::kSortReduceScan, rtg::kSortCoop}) {
        if (mode == rtg::kSortCoop && num_sms > 0 &&
            !rtg::sort_coop_fits(N, bits, items, num_sms, key64))
          continue;
        rtg::SortConfig c;
        c.bits = bits;
        c.items = items;
        c.mode = mode;
        v.push_back(c);
      }
  return v;
}

// Number after `"name": ` in a line of our own cache format (no nesting, no escapes).
bool field(const std::string& line, const char* name, double* v) {
  const std::string pat = std::string("\"") + name + "\":";
  const size_t at = line.find(pat);
  if (at == std::string::npos) return false;
  *v = std::strtod(line.c_str() + at + pat.size(), nullptr);
  return true;
}

bool field_str(const std::string& line, const char* name, std::string* v) {
  const std::string pat = std::string("\"") + name + "\": \"";
  const size_t at = line.find(pat);
  if (at == std::string::npos) return false;
  const size_t b = at + pat.size(), e = line.find('"', b);
  if (e == std::string::npos) return false;
  *v = line.substr(b, e - b);
  return true;
}

bool valid_cfg(const rtg::SortConfig& c) {
  const bool bits_ok = std::find(std::begin(rtg::kSortBitsChoices), std::end(rtg::kSortBitsChoices),
                                 c.bits) != std::end(rtg::kSortBitsChoices);
  const bool items_ok = std::find(std::begin(rtg::kSortItemsChoices),
                                  std::end(rtg::kSortItemsChoices),
                                  c.items) != std::end(rtg::kSortItemsChoices);
  return bits_ok && items_ok &&
         (c.mode == rtg::kSortLookback || c.mode == rtg::kSortReduceScan ||
          c.mode == rtg::kSortCoop);
}

// Reads the cache file into `out` (entries of this device only).
void read_cache(const std::string& path, const std::string& device,
                std::map<SortKey, TuneEntry>* out) {
  FILE* f = std::fopen(path.c_str(), "r");
  if (!f) return;
  char buf[512];
  while (std::fgets(buf, sizeof buf, f)) {
    const std::string line(buf);
    std::string dev;
    double el, kb, bits, items, mode, us;
    if (!field_str(line, "device", &dev) || dev != device) continue;
    if (!field(line, "elements", &el) || !field(line, "key_bits", &kb) ||
        !field(line, "bits", &bits) || !field(line, "items", &items) ||
        !field(line, "mode", &mode) || !field(line, "us", &us))
      continue;
    TuneEntry e;
    e.cfg.bits = (int)bits;
    e.cfg.items = (int)items;
    e.cfg.mode = (int)mode;
    e.us = us;
    if (valid_cfg(e.cfg)) (*out)[SortKey((long long)el, (int)kb)] = e;
  }
  std::fclose(f);
}

// Merges the context's entries into the cache file (write to a temporary, then rename).
void save_cache(rtg_ctx* c) {
  if (c->tune_path.empty()) return;
  std::map<SortKey, TuneEntry> all;
  read_cache(c->tune_path, c->device_name, &all);
  for (const auto& kv : c->sort_tune) all[kv.first] = kv.second;
  // keep other devices' lines as they are
  std::vector<std::string> other;
  if (FILE* f = std::fopen(c->tune_path.c_str(), "r")) {
    char buf[512];
    while (std::fgets(buf, sizeof buf, f)) {
      const std::string line(buf);
      std::string dev;
      if (field_str(line, "device", &dev) && dev != c->device_name) {
        std::string l = line;
        while (!l.empty() && (l.back() == '\n' || l.back() == ',')) l.pop_back();
        other.push_back(l);
      }
    }
    std::fclose(f);
  }
  const std::string tmp = c->tune_path + ".tmp" + std::to_string((long long)(uintptr_t)c);
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  std::fprintf(f, "{\"rtg_sort_tune\": 1, \"entries\": [\n");
  std::vector<std::string> lines = other;
  for (const auto& kv : all) {
    char line[400];
    std::snprintf(line, sizeof line,
                  "{\"device\": \"%s\", \"elements\": %lld, \"key_bits\": %d, \"bits\": %d, "
                  "\"items\": %d, \"mode\": %d, \"us\": %.2f}",
                  c->device_name.c_str(), kv.first.first, kv.first.second, kv.second.cfg.bits,
                  kv.second.cfg.items, kv.second.cfg.mode, kv.second.us);
    lines.push_back(line);
  }
  for (size_t i = 0; i < lines.size(); ++i)
    std::fprintf(f, "%s%s\n", lines[i].c_str(), i + 1 < lines.size() ? "," : "");
  std::fprintf(f, "]}\n");
  std::fclose(f);
  std::rename(tmp.c_str(), c->tune_path.c_str());
}

}  // namespace

rtg::SortConfig sort_default(long long N, int num_sms) {
  rtg::SortConfig c;
  c.bits = 8;
  c.items = 8;
  c.mode = rtg::sort_tiles_for(N, 8) <= (size_t)(3 * num_sms) ? rtg::kSortLookback
                                                               : rtg::kSortReduceScan;
  return c;
}

size_t sort_scratch_bytes(long long N, const rtg::SortConfig& cfg) {
  const size_t words = rtg::sort_tiles_for(N, cfg.items) * ((size_t)1 << cfg.bits);
  return words * (cfg.mode == rtg::kSortLookback ? 8 : 4);
}

size_t sort_scratch_bytes_max(long long N) {
  size_t m = 0;
  for (const auto& c : candidates()) m = std::max(m, sort_scratch_bytes(N, c));
  return m;
}

void tune_load(rtg_ctx* c) {
  const char* p = std::getenv("RTG_TUNE_CACHE");
  c->tune_path = p ? p : "";
  const char* off = std::getenv("RTG_AUTOTUNE");
  c->autotune = !(off && std::strcmp(off, "0") == 0);
  // in-cell candidates above which the enumeration knobs keep their defaults
  if (const char* v = std::getenv("RTG_TUNE_PAIRS_MAX_CAND")) {
    const double x = std::atof(v);
    if (x > 0.0) c->tune_pairs_max_cand = x;
  }
  c->sort_forced = false;
  if (const char* v = std::getenv("RTG_SORT_VARIANT")) {
    // "bits,items,mode": one variant for every sort of this context (no measurement)
    rtg::SortConfig f;
    if (std::sscanf(v, "%d,%d,%d", &f.bits, &f.items, &f.mode) == 3 && valid_cfg(f)) {
      c->sort_forced = true;
      c->sort_force = f;
    }
  }
  if (!c->tune_path.empty()) read_cache(c->tune_path, c->device_name, &c->sort_tune);
}

rtg_status tune_sort(rtg_ctx* c, rtg::BuildArgs& a, long long N, int key_bits,
                     rtg::SortConfig* out) {
  std::vector<rtg::SortConfig> cands = candidates(N, a.num_sms, a.key64);
  if (a.cell_major) {
    // a cell-major sort runs 8-bit digits in separate passes (its last pass rebases the keys)
    std::vector<rtg::SortConfig> keep;
    for (const rtg::SortConfig& cfg : cands)
      if (cfg.mode != rtg::kSortCoop && cfg.bits == 8) keep.push_back(cfg);
    cands.swap(keep);
  }
  const size_t nc = cands.size();
  std::vector<cudaEvent_t> ev(2 * nc, nullptr);
  std::vector<cudaGraphExec_t> exec(nc, nullptr);
  auto release = [&]() {
    for (auto& x : exec)
      if (x) cudaGraphExecDestroy(x);
    for (auto& x : ev)
      if (x) cudaEventDestroy(x);
  };
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      release();
      return fail(c, RTG_E_CUDA, "tune: cudaEventCreate failed");
    }
  const cudaStream_t st = c->stream;
  const rtg::BuildArgs base = a;
  // one trial of candidate i: the keys (the sort consumes its input buffers), then the sort
  // between two event records; inside a capture the records become event nodes
  auto trial = [&](size_t i, bool captured) {
    const rtg::SortConfig& cfg = cands[i];
    rtg::BuildArgs b = base;
    b.sort_bits = cfg.bits;
    b.sort_items = cfg.items;
    b.sort_mode = cfg.mode;
    b.passes = rtg::sort_passes_for(key_bits, cfg.bits);
    cudaMemsetAsync(&b.st->sort_tiles[0], 0, sizeof(b.st->sort_tiles), st);
    cudaMemsetAsync(&b.st->coop_count, 0, 2 * sizeof(unsigned int), st);
    rtg::launch_keys(b, st);
    if (captured) cudaEventRecordWithFlags(ev[2 * i], st, cudaEventRecordExternal);
    else cudaEventRecord(ev[2 * i], st);
    rtg::launch_sort(b, st);
    if (captured) cudaEventRecordWithFlags(ev[2 * i + 1], st, cudaEventRecordExternal);
    else cudaEventRecord(ev[2 * i + 1], st);
  };
  if (c->use_graphs) {
    for (size_t i = 0; i < nc; ++i) {
      cudaGetLastError();
      if (cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) != cudaSuccess) break;
      trial(i, true);
      cudaGraph_t g = nullptr;
      if (cudaStreamEndCapture(st, &g) != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        continue;
      }
      if (cudaGraphInstantiate(&exec[i], g, 0) != cudaSuccess) exec[i] = nullptr;
      cudaGraphDestroy(g);
    }
    cudaGetLastError();  // a candidate that could not be captured is timed directly
  }
  std::vector<std::vector<double>> samples(nc);
  cudaError_t e = cudaSuccess;
  for (int rep = 0; rep < kTuneReps && e == cudaSuccess; ++rep) {
    for (size_t i = 0; i < nc; ++i) {
      if (exec[i]) {
        if ((e = cudaGraphLaunch(exec[i], st)) != cudaSuccess) break;
      } else {
        trial(i, false);
      }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) break;
    for (size_t i = 0; i < nc; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]) == cudaSuccess)
        samples[i].push_back((double)ms * 1e3);
    }
  }
  std::vector<double> best(cands.size());
  for (size_t i = 0; i < cands.size(); ++i) best[i] = median_of(samples[i]);
  release();
  if (e != cudaSuccess)
    return fail(c, RTG_E_CUDA, std::string("tune: ") + cudaGetErrorString(e));
  size_t k = 0;
  for (size_t i = 1; i < cands.size(); ++i)
    if (best[i] < best[k]) k = i;
  *out = cands[k];
  TuneEntry te;
  te.cfg = cands[k];
  te.us = best[k];
  c->sort_tune[SortKey(N, key_bits)] = te;
  save_cache(c);
  return RTG_OK;
}

// A first enumeration trial longer than this keeps the default knobs.
constexpr float kTunePairsTrialMaxMs = 25.0f;

rtg_status tune_pairs(rtg_ctx* c, rtg::BuildArgs& a, const rtg::SortConfig& cfg, int key_bits,
                      int* spans_per_warp, int* dense_min) {
  static const int kSpans[] = {1, 2, 4};
  static const int kDense[] = {64, 128, 256};
  constexpr int kCands = 9;
  const cudaStream_t st = c->stream;
  rtg::BuildArgs b = a;
  b.skip_tail = 0;  // every kernel of the enumeration is timed
  b.sort_bits = cfg.bits;
  b.sort_items = cfg.items;
  b.sort_mode = cfg.mode;
  b.passes = rtg::sort_passes_for(key_bits, cfg.bits);
  cudaMemsetAsync(&b.st->sort_tiles[0], 0, sizeof(b.st->sort_tiles), st);
  cudaMemsetAsync(&b.st->coop_count, 0, 2 * sizeof(unsigned int), st);
  rtg::launch_keys(b, st);
  const int sorted = rtg::launch_sort(b, st);
  std::vector<cudaEvent_t> ev(2 * kCands * kTuneReps, nullptr);
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess)
      return fail(c, RTG_E_CUDA, "tune: cudaEventCreate failed");
  {
    // one trial first: an enumeration that takes long keeps the defaults (the trials would
    // cost more than the knobs can save)
    b.spans_per_warp = kSpans[0];
    b.dense_min = kDense[0];
    rtg::reset_pairs_state(b, st);
    cudaEventRecord(ev[0], st);
    rtg::launch_pairs(b, sorted, rtg::kCount, st);
    cudaEventRecord(ev[1], st);
    float ms = 0.f;
    if (cudaEventSynchronize(ev[1]) != cudaSuccess ||
        cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess || ms > kTunePairsTrialMaxMs) {
      cudaGetLastError();
      for (auto& x : ev) cudaEventDestroy(x);
      *spans_per_warp = 0;
      *dense_min = 0;
      return RTG_OK;
    }
  }
  for (int rep = 0; rep < kTuneReps; ++rep)
    for (int k = 0; k < kCands; ++k) {
      b.spans_per_warp = kSpans[k / 3];
      b.dense_min = kDense[k % 3];
      rtg::reset_pairs_state(b, st);
      cudaEventRecord(ev[2 * (rep * kCands + k)], st);
      rtg::launch_pairs(b, sorted, rtg::kCount, st);
      cudaEventRecord(ev[2 * (rep * kCands + k) + 1], st);
    }
  cudaError_t e = cudaStreamSynchronize(st);
  std::vector<std::vector<double>> samples(kCands);
  if (e == cudaSuccess)
    for (int rep = 0; rep < kTuneReps; ++rep)
      for (int k = 0; k < kCands; ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev[2 * (rep * kCands + k)], ev[2 * (rep * kCands + k) + 1]) ==
            cudaSuccess)
          samples[k].push_back((double)ms);
      }
  double best[kCands];
  for (int k = 0; k < kCands; ++k) best[k] = median_of(samples[k]);
  for (auto& x : ev) cudaEventDestroy(x);
  if (e != cudaSuccess) return fail(c, RTG_E_CUDA, std::string("tune: ") + cudaGetErrorString(e));
  int k = 0;
  for (int q = 1; q < kCands; ++q)
    if (best[q] < best[k]) k = q;
  *spans_per_warp = kSpans[k / 3];
  *dense_min = kDense[k % 3];
  return RTG_OK;
}

}  // namespace rtghost
