// Serving loop: continuous batching of independent solve requests on one GPU.
//
// Requests (lattice, blocks, excitation set) are queued; a pool of worker
// threads, each with its own CUDA stream, takes the next admissible request
// as soon as it is free, so requests that arrive while others run start on
// the device as slots and memory free up and their kernels overlap.  Arrays
// (stored bins + factored preconditioner) stay resident between requests,
// keyed by the caller's key; admission checks the HBM footprint estimate
// against a budget and evicts idle arrays least-recently used first.  Every
// request's result is that of a stand-alone solve: the kernels reduce in a
// fixed order, so sharing the device changes timing only.
//
// The server uses only the public entry points of moma.h.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "moma.h"
#include <cuda_runtime.h>

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Resident {
  moma_array *a = nullptr;
  unsigned long long key = 0;
  int nx = 0, ny = 0, b = 0;
  bool busy = false;
  double last_used = 0;
  size_t bytes = 0;
};

struct Pending {
  moma_request r;
  unsigned long long ticket;
  double t_submit;
};

}  // namespace

struct moma_server {
  moma_server_opts o{};
  int dev = 0;
  size_t budget = 0;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Pending> queue;
  std::unordered_map<unsigned long long, moma_result> done;
  std::vector<Resident> cache;
  size_t bytes_in_use = 0;   // resident arrays + reservations of running misses
  unsigned long long next_ticket = 1;
  bool stop = false;
  moma_server_stats st{};
};

namespace {

// Arrays of the serving loop skip the launch-shape timing trials (tens of
// milliseconds for an array seen once); they take shapes tuned before in
// this process for the same shape, else the built-in heuristics.
moma_options array_opts(const moma_server *s) {
  moma_options o{};
  o.precision = s->o.precision;
  o.restart = s->o.restart;
  o.flags = MOMA_FLAG_NO_AUTOTUNE;
  return o;
}

// Pick the first admissible request (FIFO with back-fill).  Called with the
// lock held; returns the queue index or -1, and sets *slot to the cache
// entry to use (-1 = a miss that has been reserved `*reserve` bytes).
int pick(moma_server *s, int *slot, size_t *reserve) {
  for (size_t qi = 0; qi < s->queue.size(); ++qi) {
    const moma_request &r = s->queue[qi].r;
    int hit = -1, busy_same = 0;
    for (size_t ci = 0; ci < s->cache.size(); ++ci) {
      const Resident &c = s->cache[ci];
      if (c.key == r.key && c.nx == r.nx && c.ny == r.ny && c.b == r.b) {
        if (!c.busy) { hit = (int)ci; break; }
        busy_same = 1;
      }
    }
    if (hit >= 0) {
      // Workspace growth for more RHS is charged on completion.
      *slot = hit;
      *reserve = 0;
      return (int)qi;
    }
    if (busy_same) continue;  // wait for the resident copy instead of building a second one
    const moma_options ao = array_opts(s);
    const size_t need = moma_estimate_bytes(r.nx, r.ny, r.b, &ao, r.nrhs, 1);
    if (need == 0 || need > s->budget) {  // can never fit: run it so that it reports the error
      *slot = -1;
      *reserve = 0;
      return (int)qi;
    }
    // Evict idle arrays, least recently used first, until the request fits.
    while (s->bytes_in_use + need > s->budget) {
      int lru = -1;
      for (size_t ci = 0; ci < s->cache.size(); ++ci)
        if (!s->cache[ci].busy && (lru < 0 || s->cache[ci].last_used < s->cache[lru].last_used)) lru = (int)ci;
      if (lru < 0) break;
      moma_destroy(s->cache[lru].a);
      s->bytes_in_use -= s->cache[lru].bytes;
      s->cache.erase(s->cache.begin() + lru);
      s->st.evictions++;
    }
    if (s->bytes_in_use + need <= s->budget) {
      // Reserve a busy placeholder under this key: later requests with the
      // same key wait for it instead of building a second copy.
      Resident ph;
      ph.key = r.key;
      ph.nx = r.nx;
      ph.ny = r.ny;
      ph.b = r.b;
      ph.busy = true;
      s->cache.push_back(ph);
      *slot = (int)s->cache.size() - 1;
      *reserve = need;
      return (int)qi;
    }
  }
  return -1;
}

moma_status run_request(moma_array *a, bool fresh, const moma_request &r, moma_result *res) {
  moma_status stt = MOMA_OK;
  if (fresh) {
    stt = moma_set_blocks(a, r.blocks, r.blocks_dtype);
    if (stt == MOMA_OK) stt = moma_release_setup(a);
    if (stt != MOMA_OK) return stt;
  }
  moma_solve_opts so{};
  so.tol = r.tol;
  stt = moma_solve(a, r.nrhs, r.V, r.I, &so, &res->info, nullptr);
  if (stt != MOMA_OK) return stt;
  if (r.Za) stt = moma_active_impedance(a, r.nrhs, r.I, r.V, r.port_basis, r.z0 > 0 ? r.z0 : 50.0, r.Za, r.Gamma);
  return stt;
}

void worker(moma_server *s, int wi) {
  cudaSetDevice(s->dev);
  cudaStream_t stream = s->streams[wi];
  for (;;) {
    Pending p;
    int slot = -1;
    size_t reserve = 0;
    moma_array *a = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      int qi = -1;
      s->cv_work.wait(lk, [&] {
        if (s->stop) return true;
        qi = pick(s, &slot, &reserve);
        return qi >= 0;
      });
      if (s->stop && qi < 0) return;
      p = s->queue[qi];
      s->queue.erase(s->queue.begin() + qi);
      if (slot >= 0 && s->cache[slot].a) {  // resident hit
        s->cache[slot].busy = true;
        a = s->cache[slot].a;
      } else {  // miss: a reserved placeholder (or a request that can never fit)
        s->bytes_in_use += reserve;
      }
    }
    moma_result res{};
    const double t_start = now_ms();
    const bool fresh = a == nullptr;
    moma_status stt = MOMA_OK;
    if (fresh) {
      moma_options ao = array_opts(s);
      stt = moma_create_array(p.r.nx, p.r.ny, p.r.b, &ao, stream, &a);
    } else {
      stt = moma_set_stream(a, stream);
    }
    if (stt == MOMA_OK) stt = run_request(a, fresh, p.r, &res);
    const double t_end = now_ms();
    res.status = stt;
    res.resident_hit = fresh ? 0 : 1;
    res.queue_ms = t_start - p.t_submit;
    res.run_ms = t_end - t_start;
    res.total_ms = t_end - p.t_submit;
    if (stt != MOMA_OK) std::strncpy(res.message, moma_last_error(), sizeof(res.message) - 1);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (fresh) {
        s->bytes_in_use -= reserve;
        // Find this request's placeholder (indices may have shifted).
        int ph = -1;
        for (size_t ci = 0; ci < s->cache.size(); ++ci)
          if (!s->cache[ci].a && s->cache[ci].busy && s->cache[ci].key == p.r.key && s->cache[ci].nx == p.r.nx &&
              s->cache[ci].ny == p.r.ny && s->cache[ci].b == p.r.b)
            ph = (int)ci;
        if (a && stt == MOMA_OK) {
          Resident c;
          c.a = a;
          c.key = p.r.key;
          c.nx = p.r.nx;
          c.ny = p.r.ny;
          c.b = p.r.b;
          c.bytes = moma_device_bytes(a);
          c.last_used = t_end;
          if (ph >= 0) s->cache[ph] = c;
          else s->cache.push_back(c);
          s->bytes_in_use += c.bytes;
        } else {
          if (a) moma_destroy(a);
          if (ph >= 0) s->cache.erase(s->cache.begin() + ph);
        }
        s->st.misses++;
      } else {
        for (auto &c : s->cache)
          if (c.a == a) {
            c.busy = false;
            c.last_used = t_end;
            const size_t nb = moma_device_bytes(a);
            s->bytes_in_use += nb - c.bytes;
            c.bytes = nb;
          }
        s->st.hits++;
      }
      s->st.completed++;
      s->done[p.ticket] = res;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

}  // namespace

extern "C" {

moma_status moma_server_create(const moma_server_opts *opt, moma_server **out) {
  if (!out) return MOMA_ERR_ARG;
  *out = nullptr;
  moma_server *s = new moma_server();
  if (opt) s->o = *opt;
  if (s->o.slots <= 0) s->o.slots = 4;
  if (s->o.precision != MOMA_PREC_FP64) s->o.precision = MOMA_PREC_MIXED;
  if (cudaGetDevice(&s->dev) != cudaSuccess) {
    delete s;
    return MOMA_ERR_CUDA;
  }
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  s->budget = s->o.max_device_bytes ? s->o.max_device_bytes : (size_t)(0.7 * (double)fr);
  for (int i = 0; i < s->o.slots; ++i) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto x : s->streams) cudaStreamDestroy(x);
      delete s;
      return MOMA_ERR_CUDA;
    }
    s->streams.push_back(st);
  }
  for (int i = 0; i < s->o.slots; ++i) s->workers.emplace_back(worker, s, i);
  *out = s;
  return MOMA_OK;
}

moma_status moma_server_submit(moma_server *s, const moma_request *r, unsigned long long *ticket) {
  if (!s || !r || !ticket) return MOMA_ERR_ARG;
  if (r->nx < 1 || r->ny < 1 || r->b < 1 || r->nrhs < 1 || !r->V || !r->I || !r->blocks) return MOMA_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    *ticket = s->next_ticket++;
    s->queue.push_back(Pending{*r, *ticket, now_ms()});
    s->st.submitted++;
  }
  s->cv_work.notify_all();
  return MOMA_OK;
}

moma_status moma_server_wait(moma_server *s, unsigned long long ticket, double timeout_s, moma_result *out) {
  if (!s || !out) return MOMA_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  const auto pred = [&] { return s->done.count(ticket) > 0; };
  if (timeout_s < 0) s->cv_done.wait(lk, pred);
  else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) return MOMA_ERR_TIMEOUT;
  *out = s->done[ticket];
  s->done.erase(ticket);
  return MOMA_OK;
}

moma_status moma_server_get_stats(moma_server *s, moma_server_stats *out) {
  if (!s || !out) return MOMA_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->resident_arrays = 0;
  for (auto &c : s->cache) out->resident_arrays += c.a ? 1 : 0;
  out->resident_bytes = s->bytes_in_use;
  out->budget_bytes = s->budget;
  out->queued = (int)s->queue.size();
  return MOMA_OK;
}

void moma_server_destroy(moma_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->queue.clear();
  }
  s->cv_work.notify_all();
  for (auto &t : s->workers) t.join();
  for (auto &c : s->cache)
    if (c.a) moma_destroy(c.a);
  for (auto st : s->streams) cudaStreamDestroy(st);
  delete s;
}

}  // extern "C"

// ------------------------------------------------------ ragged batches ----
// Independent problems of uneven sizes (different lattices, frequencies,
// RHS sets) run concurrently: `workers` host threads, each with its own
// non-blocking stream, take the next problem index; each array is bound to
// the worker's stream for its call and handed back to its own stream after.
namespace {

template <typename F>
moma_status run_batch(int n, moma_array *const *arrays, int workers, moma_status *statuses, F &&body) {
  if (n < 0 || (n > 0 && !arrays)) return MOMA_ERR_ARG;
  if (n == 0) return MOMA_OK;
  if (workers <= 0) workers = 8;
  if (workers > n) workers = n;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MOMA_ERR_CUDA;
  std::vector<cudaStream_t> streams(workers, nullptr);
  for (auto &st : streams)
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return MOMA_ERR_CUDA;
  std::vector<moma_status> stv(n, MOMA_OK);
  std::mutex mu;
  int next = 0;
  std::vector<std::thread> th;
  for (int w = 0; w < workers; ++w)
    th.emplace_back([&, w] {
      cudaSetDevice(dev);
      for (;;) {
        int i;
        {
          std::lock_guard<std::mutex> lk(mu);
          if (next >= n) return;
          i = next++;
        }
        moma_array *a = arrays[i];
        void *own = moma_array_stream(a);
        moma_status st = moma_set_stream(a, streams[w]);
        if (st == MOMA_OK) st = body(i, a);
        const moma_status back = moma_set_stream(a, own);
        stv[i] = st != MOMA_OK ? st : back;
      }
    });
  for (auto &t : th) t.join();
  for (auto st : streams) cudaStreamDestroy(st);
  moma_status first = MOMA_OK;
  for (int i = 0; i < n; ++i) {
    if (statuses) statuses[i] = stv[i];
    if (first == MOMA_OK && stv[i] != MOMA_OK) first = stv[i];
  }
  return first;
}

}  // namespace

extern "C" moma_status moma_set_blocks_batch(int n, moma_array *const *arrays, const void *const *blocks,
                                             const int *dtypes, int release_setup, int workers,
                                             moma_status *statuses) {
  if (n > 0 && (!blocks || !dtypes)) return MOMA_ERR_ARG;
  return run_batch(n, arrays, workers, statuses, [&](int i, moma_array *a) {
    moma_status st = moma_set_blocks(a, blocks[i], dtypes[i]);
    if (st == MOMA_OK && release_setup) st = moma_release_setup(a);
    return st;
  });
}

extern "C" moma_status moma_solve_batch(int n, moma_array *const *arrays, const int *nrhs, const void *const *V,
                                        void *const *I, const moma_solve_opts *opts, moma_solve_info *infos,
                                        int workers, moma_status *statuses) {
  if (n > 0 && (!nrhs || !V || !I)) return MOMA_ERR_ARG;
  return run_batch(n, arrays, workers, statuses, [&](int i, moma_array *a) {
    return moma_solve(a, nrhs[i], V[i], I[i], opts, infos ? &infos[i] : nullptr, nullptr);
  });
}
