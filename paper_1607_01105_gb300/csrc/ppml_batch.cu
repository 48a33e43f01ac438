// Host side of the batched independent 1D problems (ppml_batch_*): instance metadata, the
// work plan (which instances are split over a two-CTA cluster, largest-first order) and
// the persistent launch (kernels in ppml_batch.cuh).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/ppml.h"
#include "ppml_internal.h"
#include "ppml_launch.h"

using namespace ppml;

struct ppml_batch {
  int n_inst, dtype;
  long long total;
  double gamma, cfl;
  std::vector<int> ncells;
  InstDev* inst;
  int* order;   // one-CTA launch: the instances, largest first
  int2* items;  // cluster launch: the work items, largest first
  // plans replaced by ppml_batch_set_split: kept until ppml_batch_free, so that launches in
  // flight and captured graphs keep reading the plan they were launched with
  std::vector<void*> retired;
  int threads;  // CTA size of the launch: 256, 512 or 1024 (ppml_batch_tune / _set_threads)
  int split_min;         // instances of at least this many cells are split over a CTA pair
  int n_items, n_split;  // cluster launch: items, of which split instances (0: one-CTA launch)
  int nlmax, nmax;       // largest half of a split instance; largest one-CTA instance
  size_t smem;           // shared memory of a launch; smem_df with low parts (FP32)
  size_t smem_df;
  int max_smem;          // the device's opt-in limit per CTA
};

namespace {
constexpr int kBatchSizes[3] = {256, 512, 1024};
constexpr int kSplitFloor = 64;  // smallest instance a CTA pair may take

// Shared memory of one CTA: four fields (and for a double-float batch the three low parts)
// padded by `pad` on each side and `nface` face arrays of `faces` values.
size_t batch_smem(int cells, int pad, int nface, int nlo, int faces, size_t elt) {
  return ((4 + (size_t)nlo) * (size_t)(cells + 2 * pad) + (size_t)nface * faces) * elt;
}

// Work plan for b->split_min (ppml_batch_plan): with no instance split, one CTA per
// instance (largest first); else one cluster of two CTAs per work item, ordered largest
// first.  Sizes the launch's shared memory and copies the plan to new device buffers; the
// previous plan's buffers are retired (kept until the handle is freed), so a launch in
// flight or a captured graph never sees a half-written plan or a plan that does not match
// its shared-memory size.
int plan_batch(ppml_batch* b) {
  const size_t elt = b->dtype == PPML_F64 ? 8 : 4;
  const int nface = b->dtype == PPML_F64 ? kBatchFaceArrays<double> : kBatchFaceArrays<float>;
  const int nlo = b->dtype == PPML_F64 ? 0 : kBatchLoArrays;
  std::vector<int> items(2 * (size_t)b->n_inst), order(b->n_inst);
  int n_items = 0;
  int rc = ppml_batch_plan(b->n_inst, b->ncells.data(), b->split_min, items.data(), &n_items,
                           order.data());
  if (rc) return rc;
  int nlmax = 0, nmax = 0, n_split = 0;
  for (int i = 0; i < b->n_inst; i++) {
    if (n_items > 0 && b->split_min > 0 && b->ncells[i] >= b->split_min) {
      nlmax = std::max(nlmax, b->ncells[i] - b->ncells[i] / 2);
      n_split++;
    } else {
      nmax = std::max(nmax, b->ncells[i]);
    }
  }
  auto smem_for = [&](int lo_arrays) {
    const size_t a = n_split ? batch_smem(nlmax, kPairHalo, nface, lo_arrays, nlmax + 8, elt) : 0;
    const size_t c = nmax ? batch_smem(nmax, kBatchGhost, nface, lo_arrays, nmax + 1, elt) : 0;
    return std::max(a, c);
  };
  const size_t smem = smem_for(0), smem_df = smem_for(nlo);
  int dev = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem + 1024 > (size_t)maxsm)
    return ppml_fail(PPML_E_INVAL,
                     "largest instance needs %zu bytes of shared memory (> %d): %d cells on one "
                     "CTA, %d cells per CTA of a split one",
                     smem, maxsm, nmax, nlmax);
  int* d_order = nullptr;
  int2* d_items = nullptr;
  if (cudaMalloc(&d_order, sizeof(int) * b->n_inst) != cudaSuccess ||
      cudaMalloc(&d_items, sizeof(int2) * b->n_inst) != cudaSuccess) {
    if (d_order) cudaFree(d_order);
    return ppml_fail(PPML_E_NOMEM, "cudaMalloc of the batch work plan failed");
  }
  const cudaError_t e =
      n_items > 0
          ? cudaMemcpy(d_items, items.data(), sizeof(int2) * n_items, cudaMemcpyHostToDevice)
          : cudaMemcpy(d_order, order.data(), sizeof(int) * b->n_inst, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d_order);
    cudaFree(d_items);
    return ppml_fail(PPML_E_CUDA, "batch plan copy: %s", cudaGetErrorString(e));
  }
  if (b->order) b->retired.push_back(b->order);
  if (b->items) b->retired.push_back(b->items);
  b->order = d_order;
  b->items = d_items;
  b->n_items = n_items;
  b->n_split = n_split;
  b->nlmax = nlmax;
  b->nmax = nmax;
  b->smem = smem;
  b->smem_df = smem_df;
  b->max_smem = maxsm;
  return PPML_OK;
}

template <typename T>
int launch_typed_t(ppml_batch* b, void* const state[4], void* const lo[3], InstDev* inst,
                   int max_steps, int threads, cudaStream_t st) {
  T* f[4] = {(T*)state[0], (T*)state[1], (T*)state[2], (T*)state[3]};
  BatchLo<T> L;
  for (int q = 0; q < 3; q++) L.p[q] = lo ? (T*)lo[q] : nullptr;
  const size_t smem = lo ? b->smem_df : b->smem;
  if (smem + 1024 > (size_t)b->max_smem)
    return ppml_fail(PPML_E_INVAL,
                     "with low parts the largest instance needs %zu bytes of shared memory (> %d)",
                     smem, b->max_smem);
  int rc = launch_batch_vacuum<T>(f[0], inst, b->n_inst, st);
  if (rc) return rc;
  if (b->n_items == 0)
    return launch_batch<T>(f[0], f[1], f[2], f[3], L, inst, b->order, b->gamma, b->cfl, max_steps,
                           b->nmax, b->n_inst, smem, threads, st);
  return launch_batch_cluster<T>(f[0], f[1], f[2], f[3], L, inst, b->items, b->gamma, b->cfl,
                                 max_steps, b->nlmax, b->nmax, b->n_items, smem, threads, st);
}

void release_batch(ppml_batch* b) {
  if (b->inst) cudaFree(b->inst);
  if (b->order) cudaFree(b->order);
  if (b->items) cudaFree(b->items);
  for (void* p : b->retired) cudaFree(p);
  delete b;
}

int launch_typed(ppml_batch* b, void* const state[4], void* const lo[3], InstDev* inst,
                 int max_steps, int threads, cudaStream_t st) {
  return b->dtype == PPML_F64
             ? launch_typed_t<double>(b, state, lo, inst, max_steps, threads, st)
             : launch_typed_t<float>(b, state, lo, inst, max_steps, threads, st);
}

int check_state(const ppml_batch* b, void* const state[4], void* const lo[3]) {
  if (!state) return ppml_fail(PPML_E_INVAL, "state is NULL");
  for (int f = 0; f < 4; f++) {
    if (!state[f]) return ppml_fail(PPML_E_INVAL, "state field %d is NULL", f);
    if (((uintptr_t)state[f]) & 15u) return ppml_fail(PPML_E_INVAL, "state field %d misaligned", f);
  }
  if (lo) {
    if (b->dtype != PPML_F32) return ppml_fail(PPML_E_INVAL, "low parts are for FP32 batches only");
    for (int f = 0; f < 3; f++) {
      if (!lo[f]) return ppml_fail(PPML_E_INVAL, "low part %d is NULL (pass lo = NULL for none)", f);
      if (((uintptr_t)lo[f]) & 15u) return ppml_fail(PPML_E_INVAL, "low part %d misaligned", f);
      for (int q = 0; q < 4; q++)
        if (lo[f] == state[q]) return ppml_fail(PPML_E_INVAL, "low part %d aliases a field", f);
    }
  }
  return PPML_OK;
}

// Copy the instances' metadata to the host; counts the stopped and the flagged ones.
int read_instances(const ppml_batch* b, std::vector<InstDev>& hi, int* n_done, int* n_bad,
                   cudaStream_t st) {
  hi.resize(b->n_inst);
  if (cudaMemcpyAsync(hi.data(), b->inst, sizeof(InstDev) * b->n_inst, cudaMemcpyDeviceToHost,
                      st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ppml_fail(PPML_E_CUDA, "batch status: %s", cudaGetErrorString(cudaGetLastError()));
  int d = 0, nb = 0;
  for (auto& x : hi) {
    d += x.done && !x.bad;
    nb += x.bad;
  }
  if (n_done) *n_done = d;
  if (n_bad) *n_bad = nb;
  return PPML_OK;
}
}  // namespace

extern "C" int ppml_batch_plan(int n_inst, const int* ncells, int split_min, int* items,
                               int* n_items, int* order) {
  ppml_clear_error();
  if (n_inst < 1 || !ncells || !items || !n_items)
    return ppml_fail(PPML_E_INVAL, "need n_inst >= 1 and non-NULL ncells, items, n_items");
  if (split_min != 0 && split_min < kSplitFloor)
    return ppml_fail(PPML_E_INVAL, "split_min = %d: 0 (no split) or >= %d", split_min, kSplitFloor);
  std::vector<int> split, rest;
  for (int i = 0; i < n_inst; i++)
    (split_min > 0 && ncells[i] >= split_min ? split : rest).push_back(i);
  auto by_size = [&](int x, int y) { return ncells[x] > ncells[y]; };
  std::stable_sort(split.begin(), split.end(), by_size);
  std::stable_sort(rest.begin(), rest.end(), by_size);
  *n_items = 0;
  if (split.empty()) {
    if (order)
      for (int k = 0; k < n_inst; k++) order[k] = rest[k];
    return PPML_OK;
  }
  // (size of the item's largest instance, a, b), largest first; ties keep split items
  // ahead of whole ones and the instances' order
  std::vector<std::pair<int, std::pair<int, int>>> keyed;
  for (int i : split) keyed.push_back({ncells[i], {i, kItemSplit}});
  for (size_t k = 0; k < rest.size(); k += 2)
    keyed.push_back({ncells[rest[k]], {rest[k], k + 1 < rest.size() ? rest[k + 1] : -1}});
  std::stable_sort(keyed.begin(), keyed.end(),
                   [](const std::pair<int, std::pair<int, int>>& x,
                      const std::pair<int, std::pair<int, int>>& y) { return x.first > y.first; });
  for (size_t k = 0; k < keyed.size(); k++) {
    items[2 * k] = keyed[k].second.first;
    items[2 * k + 1] = keyed[k].second.second;
  }
  *n_items = (int)keyed.size();
  return PPML_OK;
}

extern "C" int ppml_batch_init(int n_inst, const int* ncells, const double* h,
                               const double* t_end, double gamma, double cfl,
                               double vacuum_frac, int dtype, ppml_batch** out) {
  ppml_clear_error();
  if (!out) return ppml_fail(PPML_E_INVAL, "out is NULL");
  *out = nullptr;
  if (n_inst < 1 || !ncells || !h || !t_end)
    return ppml_fail(PPML_E_INVAL, "need n_inst >= 1 and non-NULL ncells, h, t_end");
  if (!(gamma > 1.0)) return ppml_fail(PPML_E_INVAL, "gamma = %g must be > 1", gamma);
  if (!(cfl > 0.0 && cfl < 1.0)) return ppml_fail(PPML_E_INVAL, "cfl = %g not in (0,1)", cfl);
  if (dtype != PPML_F32 && dtype != PPML_F64) return ppml_fail(PPML_E_INVAL, "bad dtype %d", dtype);
  if (!(vacuum_frac > 0.0)) vacuum_frac = 1e-5;
  std::vector<InstDev> hi(n_inst);
  long long off = 0;
  int nmax = 0;
  for (int i = 0; i < n_inst; i++) {
    if (ncells[i] < 4) return ppml_fail(PPML_E_INVAL, "instance %d has %d cells (< 4)", i, ncells[i]);
    if (!(h[i] > 0.0) || !(t_end[i] > 0.0))
      return ppml_fail(PPML_E_INVAL, "instance %d: h and t_end must be positive", i);
    hi[i].off = off;
    hi[i].n = ncells[i];
    hi[i].steps = 0;
    hi[i].h = h[i];
    hi[i].t_end = t_end[i];
    hi[i].t = 0.0;
    hi[i].rho_vac = -vacuum_frac;  // fixed at the first step from the mean density
    hi[i].done = 0;
    hi[i].bad = 0;
    off += ncells[i];
    nmax = std::max(nmax, ncells[i]);
  }
  ppml_batch* b = new (std::nothrow) ppml_batch();
  if (!b) return ppml_fail(PPML_E_NOMEM, "host allocation failed");
  b->n_inst = n_inst;
  b->dtype = dtype;
  b->total = off;
  b->gamma = gamma;
  b->cfl = cfl;
  b->ncells.assign(ncells, ncells + n_inst);
  b->threads = 512;
  // default split: the instances within 1/8 of the largest size take a CTA pair, so the
  // longest runs are not left to one SM each; below 1024 cells the per-step exchange
  // costs more than the halved work saves
  b->split_min = std::max(1024, (7 * nmax + 7) / 8);
  int rc = PPML_OK;
  if (cudaMalloc(&b->inst, sizeof(InstDev) * n_inst) != cudaSuccess)
    rc = ppml_fail(PPML_E_NOMEM, "cudaMalloc of batch metadata failed");
  else if (cudaMemcpy(b->inst, hi.data(), sizeof(InstDev) * n_inst, cudaMemcpyHostToDevice) !=
           cudaSuccess)
    rc = ppml_fail(PPML_E_CUDA, "batch init copy: %s", cudaGetErrorString(cudaGetLastError()));
  else
    rc = plan_batch(b);
  if (rc) {  // release without clearing the failure's message
    cudaGetLastError();
    release_batch(b);
    return rc;
  }
  *out = b;
  return PPML_OK;
}

extern "C" int ppml_batch_step(ppml_batch* b, void* const state[4], void* const lo[3],
                               int max_steps, int* done_host, void* stream) {
  ppml_clear_error();
  if (!b) return ppml_fail(PPML_E_INVAL, "batch is NULL");
  int rc = check_state(b, state, lo);
  if (rc) return rc;
  if (max_steps < 0) return ppml_fail(PPML_E_INVAL, "max_steps < 0");
  cudaStream_t st = (cudaStream_t)stream;
  rc = launch_typed(b, state, lo, b->inst, max_steps, b->threads, st);
  if (rc) return rc;
  if (done_host) {
    std::vector<InstDev> hi;
    int n_bad = 0;
    rc = read_instances(b, hi, done_host, &n_bad, st);
    if (rc) return rc;
    if (n_bad)
      return ppml_fail(PPML_E_NONPHYSICAL, "%d instance(s) stopped on a non-physical state "
                                           "(ppml_batch_status names them)", n_bad);
  }
  return PPML_OK;
}

extern "C" int ppml_batch_set_threads(ppml_batch* b, int threads) {
  ppml_clear_error();
  if (!b) return ppml_fail(PPML_E_INVAL, "batch is NULL");
  for (int s : kBatchSizes)
    if (s == threads) {
      b->threads = threads;
      return PPML_OK;
    }
  return ppml_fail(PPML_E_INVAL, "threads = %d is not 256, 512 or 1024", threads);
}

extern "C" int ppml_batch_set_split(ppml_batch* b, int min_cells) {
  ppml_clear_error();
  if (!b) return ppml_fail(PPML_E_INVAL, "batch is NULL");
  if (min_cells != 0 && min_cells < kSplitFloor)
    return ppml_fail(PPML_E_INVAL, "min_cells = %d: 0 (no pairs) or >= %d", min_cells, kSplitFloor);
  const int old = b->split_min;
  b->split_min = min_cells;
  const int rc = plan_batch(b);  // the current plan stays in place if this fails
  if (rc) b->split_min = old;
  return rc;
}

extern "C" int ppml_batch_tune(ppml_batch* b, void* const state[4], int trial_steps,
                               int* threads_out, double ms_out[3], void* stream) {
  ppml_clear_error();
  if (!b) return ppml_fail(PPML_E_INVAL, "batch is NULL");
  int rc = check_state(b, state, nullptr);
  if (rc) return rc;
  if (trial_steps < 1) return ppml_fail(PPML_E_INVAL, "trial_steps = %d must be >= 1", trial_steps);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t elt = b->dtype == PPML_F64 ? 8 : 4;
  // scratch copies: the trials advance these, never the caller's state or the batch's times
  void* scratch[4] = {nullptr, nullptr, nullptr, nullptr};
  InstDev* inst = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double best_ms = 0.0;
  int best = b->threads;
  rc = PPML_OK;
  for (int f = 0; f < 4 && rc == PPML_OK; f++)
    if (cudaMalloc(&scratch[f], elt * (size_t)b->total) != cudaSuccess)
      rc = ppml_fail(PPML_E_NOMEM, "tuning scratch state");
  if (rc == PPML_OK && cudaMalloc(&inst, sizeof(InstDev) * b->n_inst) != cudaSuccess)
    rc = ppml_fail(PPML_E_NOMEM, "tuning scratch metadata");
  if (rc == PPML_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    rc = ppml_fail(PPML_E_CUDA, "cudaEventCreate failed");
  for (int k = 0; k < 3 && rc == PPML_OK; k++) {
    const int threads = kBatchSizes[k];
    float best_k = 0.f;
    for (int rep = 0; rep < 2 && rc == PPML_OK; rep++) {  // the first repetition also warms up
      for (int f = 0; f < 4; f++)
        if (cudaMemcpyAsync(scratch[f], state[f], elt * (size_t)b->total, cudaMemcpyDeviceToDevice,
                            st) != cudaSuccess)
          rc = ppml_fail(PPML_E_CUDA, "tuning copy: %s", cudaGetErrorString(cudaGetLastError()));
      if (rc == PPML_OK && cudaMemcpyAsync(inst, b->inst, sizeof(InstDev) * b->n_inst,
                                           cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        rc = ppml_fail(PPML_E_CUDA, "tuning copy: %s", cudaGetErrorString(cudaGetLastError()));
      if (rc) break;
      cudaEventRecord(e0, st);
      rc = launch_typed(b, scratch, nullptr, inst, trial_steps, threads, st);
      if (rc) break;
      cudaEventRecord(e1, st);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        rc = ppml_fail(PPML_E_CUDA, "tuning timing: %s", cudaGetErrorString(cudaGetLastError()));
      if (rep == 0 || ms < best_k) best_k = ms;
    }
    if (rc) break;
    if (ms_out) ms_out[k] = best_k;
    if (k == 0 || best_k < best_ms) {
      best_ms = best_k;
      best = threads;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  for (int f = 0; f < 4; f++)
    if (scratch[f]) cudaFree(scratch[f]);
  if (inst) cudaFree(inst);
  if (rc) return rc;
  b->threads = best;
  if (threads_out) *threads_out = best;
  return PPML_OK;
}

extern "C" int ppml_batch_status(ppml_batch* b, double* t_host, int* steps_host,
                                 unsigned* flags_host, void* stream) {
  ppml_clear_error();
  if (!b) return ppml_fail(PPML_E_INVAL, "batch is NULL");
  std::vector<InstDev> hi;
  int n_bad = 0;
  int rc = read_instances(b, hi, nullptr, &n_bad, (cudaStream_t)stream);
  if (rc) return rc;
  for (int i = 0; i < b->n_inst; i++) {
    if (t_host) t_host[i] = hi[i].t;
    if (steps_host) steps_host[i] = hi[i].steps;
    if (flags_host) flags_host[i] = hi[i].bad ? PPML_FLAG_NONPHYSICAL : 0u;
  }
  if (n_bad)
    return ppml_fail(PPML_E_NONPHYSICAL, "%d instance(s) stopped on a non-physical state", n_bad);
  return PPML_OK;
}

extern "C" int ppml_batch_free(ppml_batch* b) {
  ppml_clear_error();
  if (!b) return PPML_OK;
  cudaDeviceSynchronize();
  release_batch(b);
  return PPML_OK;
}
