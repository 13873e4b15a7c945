// Batched solve of independent eigenproblems (many uneven problems at once).
//
// Every problem gets its own context, hence its own CUDA stream, device
// buffers and host-side dense state; a pool of host threads takes the
// problems in index order, so the GPU work of up to `nthreads` problems
// overlaps (a small problem leaves most SMs idle on its own) and their
// Hessenberg/Schur/reordering steps run on separate host cores.  The kernels
// are deterministic, so each problem's result is the same bits as when it is
// solved alone.

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <thread>
#include <vector>

#include "../../include/rks.h"
#include "rks_impl.h"

struct rks_batch {
  int device = 0;
  std::vector<rks_ctx*> ctx;
  std::vector<int> status;
};

namespace {

// Run f(i) for i < count on up to nthreads host threads (device `dev` current
// on each), status[i] = f(i); returns the first failing status in index
// order, else RKS_OK.
template <class F>
int for_each_parallel(int count, int nthreads, int dev, F f, std::vector<int>& status) {
  status.assign(count, RKS_OK);
  std::atomic<int> next(0);
  auto worker = [&]() {
    if (cudaSetDevice(dev) != cudaSuccess) return;
    for (int i = next.fetch_add(1); i < count; i = next.fetch_add(1)) status[i] = f(i);
  };
  const int nt = std::max(1, std::min(nthreads, count));
  std::vector<std::thread> pool;
  pool.reserve(nt - 1);
  for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
  if (next.load() < count) return RKS_ECUDA;   // a worker could not select the device
  for (int s : status)
    if (s != RKS_OK) return s;
  return RKS_OK;
}

}  // namespace

extern "C" int rks_create_batched(rks_batch** out, int count, const int64_t* n, const int32_t* const* rowptr,
                                  const int32_t* const* colind, const void* const* vals, int vals_dtype, int k,
                                  int p, int d, int which, double tol, uint64_t seed, const rks_opts* opts,
                                  int nthreads) {
  if (!out) return RKS_EINVAL;
  *out = nullptr;
  if (count < 1 || !n || !rowptr || !colind || !vals) return RKS_EINVAL;
  if (opts && (opts->stream || opts->u1)) return RKS_EINVAL;   // per-problem streams and start vectors
  rks_batch* b = new (std::nothrow) rks_batch();
  if (!b) return RKS_ENOMEM;
  if (cudaGetDevice(&b->device) != cudaSuccess) { delete b; return RKS_ECUDA; }
  // one-time kernel attributes before any thread creates a context
  if (rks::configure_kernels() != cudaSuccess || rks::configure_df_kernels() != cudaSuccess ||
      rks::configure_tc_kernels() != cudaSuccess) {
    delete b;
    return RKS_ECUDA;
  }
  b->ctx.assign(count, nullptr);
  const int rc = for_each_parallel(count, nthreads, b->device, [&](int i) {
    return rks_create(&b->ctx[i], n[i], rowptr[i], colind[i], vals[i], vals_dtype, k, p, d, which, tol, seed, opts);
  }, b->status);
  if (rc != RKS_OK) {
    rks_destroy_batched(b);
    return rc;
  }
  *out = b;
  return RKS_OK;
}

extern "C" int rks_solve_batched(rks_batch* b, int nthreads, rks_info* infos) {
  if (!b) return RKS_EINVAL;
  const int count = (int)b->ctx.size();
  const int rc = for_each_parallel(count, nthreads, b->device, [&](int i) {
    return rks_solve(b->ctx[i], infos ? &infos[i] : nullptr);
  }, b->status);
  if (rc == RKS_ECUDA) return rc;
  // RKS_ENOCONV (partial results) only if nothing worse happened
  int worst = RKS_OK;
  for (int s : b->status) {
    if (s == RKS_OK) continue;
    if (s != RKS_ENOCONV) return s;
    worst = RKS_ENOCONV;
  }
  return worst;
}

extern "C" int rks_batch_count(const rks_batch* b) { return b ? (int)b->ctx.size() : 0; }

extern "C" rks_ctx* rks_batch_get(rks_batch* b, int i) {
  if (!b || i < 0 || i >= (int)b->ctx.size()) return nullptr;
  return b->ctx[i];
}

extern "C" int rks_batch_status(const rks_batch* b, int i) {
  if (!b || i < 0 || i >= (int)b->status.size()) return RKS_EINVAL;
  return b->status[i];
}

extern "C" void rks_destroy_batched(rks_batch* b) {
  if (!b) return;
  for (rks_ctx* c : b->ctx) rks_destroy(c);
  delete b;
}
