// Request server: admits factored-Schur solves of mixed meshes, dimensions and beta, keeps the
// per-(mesh, beta) factorisations resident on the device (LRU under a memory budget), and batches
// the right-hand sides of queued requests with the same (mesh, beta) into one multi-RHS solve.
// Requests that arrive while others run join the next batch of their key (continuous batching);
// batches of different keys run on different worker streams and overlap on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/schur.h"

namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Key {
  int dim, n0, n1, n2;
  double beta;
  bool operator<(const Key& o) const {
    if (dim != o.dim) return dim < o.dim;
    if (n0 != o.n0) return n0 < o.n0;
    if (n1 != o.n1) return n1 < o.n1;
    if (n2 != o.n2) return n2 < o.n2;
    return beta < o.beta;
  }
};

struct Request {
  long long ticket;
  Key key;
  schur_mesh mesh;
  double beta;
  const double* b;
  double* x;
  int nrhs;
  long long n;
  double t_submit, t_done = 0;
  int state = 0;  // 0 queued, 1 running, 2 done
  int status = SCHUR_OK;
  schur_stats st;
};

struct Entry {
  schur_ctx* ctx = nullptr;
  long long bytes = 0;
  int busy = 0;
  double last_use = 0;
};

// subdomain edge length in elements used by the server (the configurations' 16 in 2D, 8 in 3D)
int pick_nsub(int nel, int dim) {
  int s = dim == 2 ? 16 : 8;
  if (nel % s == 0 && nel / s >= 1) return nel / s;
  for (int t = s; t >= 2; --t)
    if (nel % t == 0) return nel / t;
  return 1;
}

}  // namespace

struct schur_server {
  schur_server_opts o;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::map<long long, std::shared_ptr<Request>> reqs;
  std::deque<std::shared_ptr<Request>> queue;  // arrival order
  std::map<Key, Entry> cache;
  long long bytes_used = 0, next_ticket = 1, completed = 0;
  // batching statistics (guarded by mu)
  long long n_batches = 0, n_batch_cols = 0, n_shared = 0, n_setups = 0;
  int inflight = 0, max_inflight = 0;
  bool stop = false;
  std::vector<std::thread> workers;

  schur_opts opts_for(const schur_mesh& m) const {
    schur_opts op;
    schur_default_opts(&op);
    for (int a = 0; a < 3; ++a) op.nsub[a] = a < m.dim ? pick_nsub(m.nel[a], m.dim) : 1;
    op.precision = o.precision;
    op.tol = o.tol;
    op.max_iter = o.max_iter;
    return op;
  }

  // right-hand-side columns of the largest batch a request can be solved in: batches hold up to
  // max_batch_rhs columns, or one request alone if it is larger
  int batch_cols(int nrhs) const { return std::max(nrhs, o.max_batch_rhs); }

  // device bytes a context for mesh m will hold (factors, operators, coarse inverse, workspace for
  // the largest batch it can serve: the solver works on at most 16 columns at a time), from
  // closed-form partition counts (no map building), or -1 for an unusable mesh
  long long estimate(const schur_mesh& m, int nrhs) const {
    if (m.dim != 2 && m.dim != 3) return -1;
    long long nsd = 1, nl = 1, ni = 1, n = 1, nco = 1, nlam = 0, L = 1;
    long long Pa[3] = {1, 1, 1}, sa[3] = {1, 1, 1};
    for (int a = 0; a < m.dim; ++a) {
      int P = pick_nsub(m.nel[a], m.dim), s = m.nel[a] / P;
      if (s < 2) return -1;
      Pa[a] = P;
      sa[a] = s;
      nsd *= P;
      nl *= s + 1;
      ni *= s - 1;
      n *= m.nel[a] - 1;
      nco *= P - 1;
      L = s + 1;
    }
    const long long nD = nl - ni - (1LL << m.dim), b = nl / L;
    // multipliers: one per interior face node of each pair of face neighbours; in 3D also six per
    // node of each subdomain edge line shared by four subdomains (fully redundant)
    for (int a = 0; a < m.dim; ++a) {
      long long f = Pa[a] - 1;
      for (int c = 0; c < m.dim; ++c)
        if (c != a) f *= Pa[c] * (sa[c] - 1);
      nlam += f;
      if (m.dim == 3) {
        long long e = 6 * Pa[a] * (sa[a] - 1);
        for (int c = 0; c < 3; ++c)
          if (c != a) e *= Pa[c] - 1;
        nlam += e;
      }
    }
    const long long cxb = o.precision == SCHUR_MIXED ? 8 : 16;
    long long ops = nsd * (L * b * b + 2 * nD * nD + 8 * nD) * cxb + nco * nco * cxb;
    // 3D mixed setup also holds the two layer-coupling arrays of the tensor-core formation
    if (m.dim == 3 && o.precision == SCHUR_MIXED) ops += 2 * nsd * L * b * b * cxb;
    const long long R = std::min(batch_cols(nrhs), 16);
    long long ws = nsd * nl * R * cxb + nlam * R * (o.max_iter + 5) * cxb + n * R * 32 + nsd * nD * R * 3 * cxb;
    return ops + ws + (64LL << 20);
  }

  // LRU eviction of idle cache entries until `need` more bytes fit; false if impossible now
  bool make_room(long long need) {
    while (bytes_used + need > (long long)o.device_mem_budget) {
      auto victim = cache.end();
      for (auto it = cache.begin(); it != cache.end(); ++it)
        if (!it->second.busy && (victim == cache.end() || it->second.last_use < victim->second.last_use)) victim = it;
      if (victim == cache.end()) return false;
      bytes_used -= victim->second.bytes;
      schur_destroy(victim->second.ctx);
      cache.erase(victim);
    }
    return true;
  }

  void worker_main() {
    cudaSetDevice(device);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    double *hb = nullptr, *hx = nullptr, *db = nullptr, *dx = nullptr;
    size_t cap = 0;
    // device bytes of this worker's b/x buffers counted in bytes_used (reserved before growing)
    long long io_reserved = 0;
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      // pick the oldest queued request whose key is not busy and whose memory (context and this
      // worker's device buffers for its largest batch) can be admitted
      std::shared_ptr<Request> head;
      Entry* ent = nullptr;
      bool need_setup = false;
      long long need = 0;
      while (!stop) {
        for (auto& r : queue) {
          const long long io = std::max(0LL, 2LL * r->n * batch_cols(r->nrhs) * (long long)sizeof(double) - io_reserved);
          auto it = cache.find(r->key);
          if (it != cache.end()) {
            if (it->second.busy) continue;
            it->second.busy = 1;  // kept out of eviction while room is made for the buffers
            const bool ok = make_room(io);
            it->second.busy = 0;
            if (!ok) continue;
            bytes_used += io;
            io_reserved += io;
            head = r;
            ent = &it->second;
            break;
          }
          long long e = estimate(r->mesh, r->nrhs);
          if (e < 0) {
            r->status = SCHUR_EINVAL;
            head = r;
            break;
          }
          if (make_room(e + io)) {
            bytes_used += io;
            io_reserved += io;
            head = r;
            need_setup = true;
            need = e;
            break;
          }
        }
        if (head) break;
        cv_work.wait(lk);
      }
      if (!head) break;
      // batch: queued requests of the same key, arrival order, up to max_batch_rhs columns
      std::vector<std::shared_ptr<Request>> batch;
      int cols = 0;
      if (head->status == SCHUR_OK) {
        for (auto& r : queue) {
          if (r->key < head->key || head->key < r->key) continue;
          if (!batch.empty() && cols + r->nrhs > o.max_batch_rhs) break;
          batch.push_back(r);
          cols += r->nrhs;
        }
      } else {
        batch.push_back(head);
      }
      for (auto& r : batch) r->state = 1;
      queue.erase(std::remove_if(queue.begin(), queue.end(), [](const std::shared_ptr<Request>& r) { return r->state == 1; }),
                  queue.end());
      if (head->status != SCHUR_OK) {
        finish(batch, head->status, nullptr);
        continue;
      }
      if (need_setup) {
        bytes_used += need;
        Entry& e = cache[head->key];
        e.bytes = need;
        e.busy = 1;
        ent = &e;
      } else {
        ent->busy = 1;
      }
      const Key key = head->key;
      ++n_batches;
      n_batch_cols += cols;
      if (batch.size() > 1) n_shared += (long long)batch.size();
      if (need_setup) ++n_setups;
      max_inflight = std::max(max_inflight, ++inflight);
      lk.unlock();
      int rc = SCHUR_OK;
      schur_ctx* ctx = ent->ctx;
      if (!ctx) {
        schur_opts op = opts_for(head->mesh);
        rc = schur_setup(&head->mesh, head->beta, &op, st, &ctx);
      }
      const long long n = head->n;
      const size_t bytes = (size_t)n * cols * sizeof(double);
      if (rc == SCHUR_OK && bytes > cap) {
        if (hb) cudaFreeHost(hb);
        if (hx) cudaFreeHost(hx);
        if (db) cudaFree(db);
        if (dx) cudaFree(dx);
        hb = hx = db = dx = nullptr;
        cap = 0;
        if (cudaMallocHost(&hb, bytes) != cudaSuccess || cudaMallocHost(&hx, bytes) != cudaSuccess ||
            cudaMalloc(&db, bytes) != cudaSuccess || cudaMalloc(&dx, bytes) != cudaSuccess)
          rc = SCHUR_ENOMEM;
        else
          cap = bytes;
      }
      schur_stats sst;
      std::memset(&sst, 0, sizeof(sst));
      if (rc == SCHUR_OK) {
        size_t off = 0;
        for (auto& r : batch) {
          std::memcpy(hb + off, r->b, sizeof(double) * n * r->nrhs);
          off += (size_t)n * r->nrhs;
        }
        cudaMemcpyAsync(db, hb, bytes, cudaMemcpyHostToDevice, st);
        rc = schur_solve(ctx, db, dx, cols, (int)n, st, &sst);
        if (rc == SCHUR_OK || rc == SCHUR_ENOTCONV) {
          cudaMemcpyAsync(hx, dx, bytes, cudaMemcpyDeviceToHost, st);
          if (cudaStreamSynchronize(st) != cudaSuccess) rc = SCHUR_ECUDA;
          off = 0;
          for (auto& r : batch) {
            std::memcpy(r->x, hx + off, sizeof(double) * n * r->nrhs);
            off += (size_t)n * r->nrhs;
          }
        }
      }
      if (rc != SCHUR_OK && rc != SCHUR_ENOTCONV)
        fprintf(stderr, "schur_server: batch of %d request(s) failed: %s: %s\n", (int)batch.size(), schur_strerror(rc),
                schur_last_error());
      lk.lock();
      --inflight;
      auto it = cache.find(key);
      if (it != cache.end()) {
        if (!it->second.ctx && ctx) it->second.ctx = ctx;
        it->second.busy = 0;
        it->second.last_use = now_ms();
        if (!it->second.ctx) {  // setup failed: release the reservation
          bytes_used -= it->second.bytes;
          cache.erase(it);
        }
      } else if (ctx) {
        schur_destroy(ctx);
      }
      finish(batch, rc, &sst);
    }
    bytes_used -= io_reserved;
    lk.unlock();
    if (hb) cudaFreeHost(hb);
    if (hx) cudaFreeHost(hx);
    if (db) cudaFree(db);
    if (dx) cudaFree(dx);
    cudaStreamDestroy(st);
  }

  // called with mu held
  void finish(std::vector<std::shared_ptr<Request>>& batch, int rc, const schur_stats* s) {
    double t = now_ms();
    for (auto& r : batch) {
      r->status = rc;
      if (s) r->st = *s;
      r->t_done = t;
      r->st.status = rc;
      r->st.ms_solve = t - r->t_submit;
      r->state = 2;
      ++completed;
    }
    cv_done.notify_all();
    cv_work.notify_all();
  }
};

extern "C" {

void schur_server_default_opts(schur_server_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->device_mem_budget = (size_t)64 << 30;
  o->workers = 4;
  o->precision = SCHUR_MIXED;
  o->tol = 1e-10;
  o->max_batch_rhs = 16;
  o->max_iter = 300;
}

int schur_server_create(const schur_server_opts* o, schur_server** out) {
  if (!o || !out || o->workers < 1 || o->workers > 64 || o->max_batch_rhs < 1 || !(o->tol > 0) ||
      (o->precision != SCHUR_FP64 && o->precision != SCHUR_MIXED))
    return SCHUR_EINVAL;
  schur_server* s = new (std::nothrow) schur_server();
  if (!s) return SCHUR_ENOMEM;
  s->o = *o;
  if (s->o.max_iter <= 0) s->o.max_iter = 300;
  cudaGetDevice(&s->device);
  for (int i = 0; i < o->workers; ++i) s->workers.emplace_back([s] { s->worker_main(); });
  *out = s;
  return SCHUR_OK;
}

int schur_submit(schur_server* s, const schur_mesh* mesh, double beta, const double* b_host, int nrhs, double* x_host,
                 long long* ticket) {
  if (!s || !mesh || !ticket || !b_host || !x_host || nrhs < 1 || !(beta > 0)) return SCHUR_EINVAL;
  long long n = schur_ndof(mesh);
  if (n <= 0) return SCHUR_EINVAL;
  auto r = std::make_shared<Request>();
  r->mesh = *mesh;
  r->key = Key{mesh->dim, mesh->nel[0], mesh->nel[1], mesh->dim == 3 ? mesh->nel[2] : 1, beta};
  r->beta = beta;
  r->b = b_host;
  r->x = x_host;
  r->nrhs = nrhs;
  r->n = n;
  r->t_submit = now_ms();
  std::memset(&r->st, 0, sizeof(r->st));
  {
    std::lock_guard<std::mutex> lk(s->mu);
    long long need = s->estimate(*mesh, nrhs);
    if (need < 0) return SCHUR_EINVAL;
    need += 2LL * n * s->batch_cols(nrhs) * (long long)sizeof(double);  // a worker's b/x buffers
    if (need > (long long)s->o.device_mem_budget) return SCHUR_EBUSY;  // can never be admitted
    r->ticket = s->next_ticket++;
    s->reqs[r->ticket] = r;
    s->queue.push_back(r);
  }
  s->cv_work.notify_all();
  *ticket = r->ticket;
  return SCHUR_OK;
}

int schur_poll(schur_server* s, long long ticket, schur_stats* st) {
  if (!s) return SCHUR_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return SCHUR_EINVAL;
  if (it->second->state != 2) return 1;
  if (st) *st = it->second->st;
  return it->second->status == SCHUR_ENOTCONV ? SCHUR_OK : it->second->status;
}

int schur_wait(schur_server* s, long long ticket, double timeout_ms, schur_stats* st) {
  if (!s) return SCHUR_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return SCHUR_EINVAL;
  auto r = it->second;
  bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), [&] { return r->state == 2; });
  if (!ok) return SCHUR_ETIMEOUT;
  if (st) *st = r->st;
  return r->status == SCHUR_ENOTCONV ? SCHUR_OK : r->status;
}

int schur_server_info(schur_server* s, schur_server_info_t* info) {
  if (!s || !info) return SCHUR_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  info->cached_contexts = (int)s->cache.size();
  info->queued = (int)s->queue.size();
  info->completed = s->completed;
  info->bytes_reserved = s->bytes_used;
  info->batches = s->n_batches;
  info->batch_columns = s->n_batch_cols;
  info->shared_requests = s->n_shared;
  info->setups = s->n_setups;
  info->max_concurrent = s->max_inflight;
  for (int i = 0; i < 3; ++i) info->reserved[i] = 0;
  return SCHUR_OK;
}

void schur_server_destroy(schur_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& kv : s->cache)
    if (kv.second.ctx) schur_destroy(kv.second.ctx);
  delete s;
}

}  // extern "C"
