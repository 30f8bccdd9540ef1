// gbdct_multi.cu - uneven-size batches of 2D transforms and the family autotuner.
//
// Batch parallelism (Section IV: independent transforms are the unit of
// parallel work): a gbdct_multi executor takes a list of 2D shapes, groups the
// transforms of equal shape into batched plans (one launch sequence per group,
// blockIdx.z over the group's transforms), and lays the transforms out in one
// packed buffer, group after group, so that each group is a dense batch.  An
// exec forks the groups onto parallel streams and joins them on the caller's
// stream; with GBDCT_MULTI_GRAPH the whole fork/join is captured once per
// (in, out, direction) as a CUDA graph and replayed by a single launch.
//
// gbdct_plan_create_tuned times every kernel family that supports a shape
// (forward + inverse with CUDA events on a private stream) and keeps the
// fastest; results are cached per process and, when GBDCT_TUNE_CACHE names a
// file, in that file (one "key family microseconds" line per entry).
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/gbdct.h"

namespace {

bool pow2_in(int64_t v, int lo, int hi) {
  if (v <= 0 || (v & (v - 1))) return false;
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return l >= lo && l <= hi;
}

gbdct_status cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return GBDCT_OK;
  return e == cudaErrorMemoryAllocation ? GBDCT_ERR_OOM : GBDCT_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Autotuner
// ---------------------------------------------------------------------------

// candidates: the kernel families, the four-step family with each split
// N1 = A * (N1 / A) of its column FFT (tile shape of the column steps), and
// the two-pass family with each strip width (column pairs per CTA)
const char* const kFamilies[] = {"tp",     "fs2",    "pair",    "seq",  "fs2/16", "fs2/32", "fs2/64", "fs2/128",
                                 "tp/1",   "tp/2",   "tp/4",    "tp/8", "tp/16",  "tp/32"};

std::mutex g_tune_mu;
std::map<std::string, std::string>* g_tune = nullptr;  // key -> family
bool g_tune_loaded = false;

std::string tune_key(int ndim, const int64_t* dims, int64_t batch, int kind) {
  char buf[160];
  int n = snprintf(buf, sizeof buf, "d%d", ndim);
  for (int i = 0; i < ndim && n < (int)sizeof buf; ++i) n += snprintf(buf + n, sizeof buf - n, "x%lld", (long long)dims[i]);
  snprintf(buf + n, sizeof buf - n, "_b%lld_k%d", (long long)batch, kind);
  return buf;
}

void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  if (!g_tune) g_tune = new std::map<std::string, std::string>();
  const char* path = getenv("GBDCT_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char key[160], fam[16];
  double us;
  while (fscanf(f, "%159s %15s %lf", key, fam, &us) == 3) (*g_tune)[key] = fam;
  fclose(f);
}

void tune_store_locked(const std::string& key, const char* fam, double us) {
  (*g_tune)[key] = fam;
  const char* path = getenv("GBDCT_TUNE_CACHE");
  if (!path || !*path) return;
  if (FILE* f = fopen(path, "a")) {
    fprintf(f, "%s %s %.3f\n", key.c_str(), fam, us);
    fclose(f);
  }
}

// Microseconds of one forward + inverse (inverse only for the inverse-only
// kinds) of `plan` on scratch buffers, best of a few runs; < 0 on error.
double time_plan(gbdct_plan_t plan, int kind, float* a, float* b, cudaStream_t s) {
  const bool fwd = kind == GBDCT_DCT2 || kind == GBDCT_DST2;
  auto run = [&]() -> gbdct_status {
    gbdct_status st = GBDCT_OK;
    if (fwd) st = gbdct_exec_forward(plan, a, b, s);
    if (st == GBDCT_OK) st = gbdct_exec_inverse(plan, fwd ? b : a, fwd ? a : b, s);
    return st;
  };
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return -1;
  }
  double best = -1;
  bool ok = run() == GBDCT_OK && cudaStreamSynchronize(s) == cudaSuccess;
  for (int r = 0; ok && r < 3; ++r) {
    ok = cudaEventRecord(e0, s) == cudaSuccess;
    for (int i = 0; ok && i < 3; ++i) ok = run() == GBDCT_OK;
    ok = ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
    float ms = 0;
    if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
      const double us = 1e3 * ms / 3;
      if (best < 0 || us < best) best = us;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ok ? best : -1;
}

}  // namespace

extern "C" {

gbdct_status gbdct_plan_create_tuned(gbdct_plan_t* out, int ndim, const int64_t* dims, int64_t batch, int kind,
                                     int dtype, char* family_out, size_t family_cap) {
  if (!out || !dims || ndim < 1 || ndim > 3 || batch < 1) return GBDCT_ERR_INVALID_ARG;
  const std::string key = tune_key(ndim, dims, batch, kind);
  std::string cached;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_load_locked();
    auto it = g_tune->find(key);
    if (it != g_tune->end()) cached = it->second;
  }
  auto report = [&](const char* fam) {
    if (family_out && family_cap) {
      strncpy(family_out, fam, family_cap - 1);
      family_out[family_cap - 1] = 0;
    }
  };
  if (!cached.empty() && gbdct_plan_create_family(out, ndim, dims, batch, kind, dtype, cached.c_str()) == GBDCT_OK) {
    report(cached.c_str());
    return GBDCT_OK;
  }
  // Validate the shape once through the default path (no timing if it fails).
  gbdct_plan_t best = nullptr;
  gbdct_status st = gbdct_plan_create_batched(&best, ndim, dims, batch, kind, dtype);
  if (st != GBDCT_OK) return st;
  int64_t elems = batch;
  for (int i = 0; i < ndim; ++i) elems *= dims[i];
  float *a = nullptr, *b = nullptr;
  cudaStream_t s = nullptr;
  cudaError_t e = cudaMalloc(&a, (size_t)elems * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&b, (size_t)elems * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(a, 0, (size_t)elems * sizeof(float));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaFree(a);
    cudaFree(b);
    gbdct_plan_destroy(best);
    return cuda_err(e);
  }
  std::string best_fam = gbdct_plan_kernel_family(best);
  double best_us = time_plan(best, kind, a, b, s);
  for (const char* fam : kFamilies) {
    if (best_fam == fam) continue;
    gbdct_plan_t p = nullptr;
    if (gbdct_plan_create_family(&p, ndim, dims, batch, kind, dtype, fam) != GBDCT_OK) continue;
    const double us = time_plan(p, kind, a, b, s);
    if (us > 0 && (best_us < 0 || us < best_us)) {
      gbdct_plan_destroy(best);
      best = p;
      best_us = us;
      best_fam = fam;
    } else {
      gbdct_plan_destroy(p);
    }
  }
  cudaStreamDestroy(s);
  cudaFree(a);
  cudaFree(b);
  if (best_us < 0) {
    gbdct_plan_destroy(best);
    return GBDCT_ERR_CUDA;
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_store_locked(key, best_fam.c_str(), best_us);
  }
  report(best_fam.c_str());
  *out = best;
  return GBDCT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Multi-shape executor
// ---------------------------------------------------------------------------

namespace {

struct Group {
  int64_t n1, n2, count, offset;  // offset in floats of the group's first transform
  gbdct_plan_t plan;
};

struct GraphEntry {
  const void* in;
  void* out;
  int inverse;
  cudaGraphExec_t exec;
};

constexpr int kMaxSide = 8;
constexpr size_t kMaxGraphs = 8;

}  // namespace

struct gbdct_multi_s {
  int device = 0, kind = 0, flags = 0;
  std::vector<Group> groups;
  std::vector<int64_t> offsets;  // per transform, in floats
  int64_t total = 0;
  std::vector<cudaStream_t> side;
  cudaStream_t capture = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  std::vector<GraphEntry> graphs;
};

namespace {

void destroy_multi(gbdct_multi_s* m) {
  if (!m) return;
  for (auto& g : m->graphs) cudaGraphExecDestroy(g.exec);
  for (auto& g : m->groups) gbdct_plan_destroy(g.plan);
  for (auto s : m->side) cudaStreamDestroy(s);
  if (m->capture) cudaStreamDestroy(m->capture);
  if (m->fork) cudaEventDestroy(m->fork);
  for (auto e : m->join) cudaEventDestroy(e);
  delete m;
}

// Fork the groups from `s` onto the side streams and join them back.
gbdct_status enqueue(gbdct_multi_s* m, bool inverse, const float* in, float* out, cudaStream_t s) {
  if (cudaEventRecord(m->fork, s) != cudaSuccess) return GBDCT_ERR_CUDA;
  const size_t nside = m->side.size();
  for (size_t i = 0; i < m->groups.size(); ++i) {
    const Group& g = m->groups[i];
    cudaStream_t cs = m->side[i % nside];
    if (cudaStreamWaitEvent(cs, m->fork, 0) != cudaSuccess) return GBDCT_ERR_CUDA;
    const gbdct_status st = inverse ? gbdct_exec_inverse(g.plan, in + g.offset, out + g.offset, cs)
                                    : gbdct_exec_forward(g.plan, in + g.offset, out + g.offset, cs);
    if (st != GBDCT_OK) return st;
    if (cudaEventRecord(m->join[i], cs) != cudaSuccess) return GBDCT_ERR_CUDA;
  }
  for (size_t i = 0; i < m->groups.size(); ++i)
    if (cudaStreamWaitEvent(s, m->join[i], 0) != cudaSuccess) return GBDCT_ERR_CUDA;
  return GBDCT_OK;
}

}  // namespace

namespace {

// Shape groups in execution order (largest transforms first), each at most
// 65535 transforms: (n1, n2, member indices).
struct LayoutGroup {
  int64_t n1, n2;
  std::vector<int> members;
};

std::vector<LayoutGroup> plan_layout(int count, const int64_t* shapes, std::vector<int64_t>* offsets,
                                     int64_t* total) {
  std::map<std::pair<int64_t, int64_t>, std::vector<int>> by_shape;
  for (int i = 0; i < count; ++i) by_shape[{shapes[2 * i], shapes[2 * i + 1]}].push_back(i);
  std::vector<std::pair<std::pair<int64_t, int64_t>, std::vector<int>>> order(by_shape.begin(), by_shape.end());
  std::stable_sort(order.begin(), order.end(), [](const auto& x, const auto& y) {
    return x.first.first * x.first.second > y.first.first * y.first.second;
  });
  std::vector<LayoutGroup> groups;
  offsets->assign(count, 0);
  int64_t off = 0;
  for (auto& kv : order) {
    const int64_t sz = kv.first.first * kv.first.second;
    for (size_t b0 = 0; b0 < kv.second.size(); b0 += 65535) {
      const size_t cnt = std::min<size_t>(65535, kv.second.size() - b0);
      LayoutGroup g{kv.first.first, kv.first.second, {}};
      for (size_t j = 0; j < cnt; ++j) {
        const int idx = kv.second[b0 + j];
        g.members.push_back(idx);
        (*offsets)[idx] = off + (int64_t)j * sz;
      }
      off += (int64_t)cnt * sz;
      groups.push_back(std::move(g));
    }
  }
  *total = off;
  return groups;
}

gbdct_status check_shapes(int count, const int64_t* shapes) {
  if (!shapes || count < 1) return GBDCT_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    if (shapes[2 * i] <= 0 || shapes[2 * i + 1] <= 0) return GBDCT_ERR_INVALID_ARG;
    if (!pow2_in(shapes[2 * i], 1, 14) || !pow2_in(shapes[2 * i + 1], 1, 14)) return GBDCT_ERR_UNSUPPORTED;
  }
  return GBDCT_OK;
}

}  // namespace

extern "C" {

int64_t gbdct_multi_layout(int count, const int64_t* shapes, int64_t* offsets, int* groups) {
  if (check_shapes(count, shapes) != GBDCT_OK) return -1;
  std::vector<int64_t> offs;
  int64_t total = 0;
  const std::vector<LayoutGroup> g = plan_layout(count, shapes, &offs, &total);
  if (offsets)
    for (int i = 0; i < count; ++i) offsets[i] = offs[i];
  if (groups) *groups = (int)g.size();
  return total;
}

gbdct_status gbdct_multi_create(gbdct_multi_t* out, int count, const int64_t* shapes, int kind, int flags) {
  if (!out || !shapes || count < 1) return GBDCT_ERR_INVALID_ARG;
  if (kind < GBDCT_DCT2 || kind > GBDCT_IDXST_IDCT) return GBDCT_ERR_INVALID_ARG;
  if (flags & ~(GBDCT_MULTI_GRAPH | GBDCT_MULTI_TUNE)) return GBDCT_ERR_INVALID_ARG;
  if (const gbdct_status cs = check_shapes(count, shapes)) return cs;
  gbdct_multi_s* m = new (std::nothrow) gbdct_multi_s();
  if (!m) return GBDCT_ERR_OOM;
  m->kind = kind;
  m->flags = flags;
  if (cudaGetDevice(&m->device) != cudaSuccess) {
    delete m;
    return GBDCT_ERR_CUDA;
  }
  // Group by shape (largest transforms first, so that they start first);
  // a group holds at most 65535 transforms (one batched plan).
  int64_t off = 0;
  const std::vector<LayoutGroup> layout = plan_layout(count, shapes, &m->offsets, &off);
  gbdct_status st = GBDCT_OK;
  for (const LayoutGroup& lg : layout) {
    const int64_t cnt = (int64_t)lg.members.size();
    Group g{lg.n1, lg.n2, cnt, m->offsets[lg.members[0]], nullptr};
    const int64_t dims[2] = {lg.n1, lg.n2};
    st = (flags & GBDCT_MULTI_TUNE) ? gbdct_plan_create_tuned(&g.plan, 2, dims, cnt, kind, GBDCT_F32, nullptr, 0)
                                    : gbdct_plan_create_batched(&g.plan, 2, dims, cnt, kind, GBDCT_F32);
    if (st != GBDCT_OK) break;
    m->groups.push_back(g);
  }
  m->total = off;
  cudaError_t e = cudaSuccess;
  if (st == GBDCT_OK) {
    const int nside = std::min<int>(kMaxSide, (int)m->groups.size());
    for (int i = 0; i < nside && e == cudaSuccess; ++i) {
      cudaStream_t s;
      e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
      if (e == cudaSuccess) m->side.push_back(s);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&m->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->fork, cudaEventDisableTiming);
    for (size_t i = 0; i < m->groups.size() && e == cudaSuccess; ++i) {
      cudaEvent_t ev;
      e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e == cudaSuccess) m->join.push_back(ev);
    }
    st = cuda_err(e);
  }
  if (st != GBDCT_OK) {
    destroy_multi(m);
    return st;
  }
  *out = m;
  return GBDCT_OK;
}

int64_t gbdct_multi_offset(gbdct_multi_t m, int index) {
  if (!m || index < 0 || index >= (int)m->offsets.size()) return -1;
  return m->offsets[index];
}

int64_t gbdct_multi_total_elems(gbdct_multi_t m) { return m ? m->total : 0; }

int gbdct_multi_group_count(gbdct_multi_t m) { return m ? (int)m->groups.size() : 0; }

const char* gbdct_multi_group_family(gbdct_multi_t m, int group) {
  if (!m || group < 0 || group >= (int)m->groups.size()) return "";
  return gbdct_plan_kernel_family(m->groups[group].plan);
}

gbdct_status gbdct_multi_exec(gbdct_multi_t m, int inverse, const void* in, void* out, void* stream) {
  if (!m || !in || !out) return GBDCT_ERR_INVALID_ARG;
  if (((uintptr_t)in & 15u) || ((uintptr_t)out & 15u)) return GBDCT_ERR_INVALID_ARG;
  if (!inverse && (m->kind == GBDCT_IDCT_IDXST || m->kind == GBDCT_IDXST_IDCT)) return GBDCT_ERR_UNSUPPORTED;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return GBDCT_ERR_CUDA;
  if (prev != m->device && cudaSetDevice(m->device) != cudaSuccess) return GBDCT_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const float* fin = static_cast<const float*>(in);
  float* fout = static_cast<float*>(out);
  gbdct_status st = GBDCT_OK;
  if (!(m->flags & GBDCT_MULTI_GRAPH)) {
    st = enqueue(m, inverse != 0, fin, fout, s);
  } else {
    cudaGraphExec_t exec = nullptr;
    for (auto& g : m->graphs)
      if (g.in == in && g.out == out && g.inverse == (inverse != 0)) exec = g.exec;
    if (!exec) {
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamBeginCapture(m->capture, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        st = enqueue(m, inverse != 0, fin, fout, m->capture);
        e = cudaStreamEndCapture(m->capture, &graph);
        if (st == GBDCT_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
      }
      if (st == GBDCT_OK) st = cuda_err(e);
      if (st == GBDCT_OK) {
        if (m->graphs.size() >= kMaxGraphs) {
          cudaGraphExecDestroy(m->graphs.front().exec);
          m->graphs.erase(m->graphs.begin());
        }
        m->graphs.push_back({in, out, inverse != 0, exec});
      }
    }
    if (st == GBDCT_OK) st = cuda_err(cudaGraphLaunch(exec, s));
  }
  if (prev != m->device) cudaSetDevice(prev);
  return st;
}

gbdct_status gbdct_multi_destroy(gbdct_multi_t m) {
  if (!m) return GBDCT_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != m->device) cudaSetDevice(m->device);
  destroy_multi(m);
  if (prev != m->device) cudaSetDevice(prev);
  return GBDCT_OK;
}

}  // extern "C"
