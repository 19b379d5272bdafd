// Serving: the request loop of include/nufft_serve.h.
//
// Policy (Scheduler, host only): FIFO admission by free execution slot and
// device-memory budget; resident plan entries keyed by request shape, reused
// when idle and large enough, destroyed least-recently-used first when a new
// entry would not fit; completion through nufft_server_complete; per-request
// time limit measured from admission.
//
// Mechanism (GpuExecutor): plan entries are nufft plans (plus scratch for
// gradient requests) on the server's device; each admitted request is
// enqueued on its slot's stream and a host callback at the end of that stream
// reports completion, so the scheduler thread never waits on the device.
//
// A least-squares gradient request (NUFFT_REQ_LSQ_GRAD) evaluates
//   loss = sum_j |c_j - y_j|^2,  c = F2_s(x) f  (Eq. (2)),
//   grad_f = 2 F1_{-s}(x) (c - y)                 (the adjoint, Sec. 1),
//   grad_x_{j,d} = 2 Re( conj(c_j - y_j) (F2_s(x) [(s i k_d) f])_j ),
// the last being the exact derivative of the exponential sum, formed as one
// more type-2 transform per dimension on the same sorted points, or (flag
// NUFFT_FLAG_XGRAD_KERNEL) taken from the first transform's interpolation
// differentiated through the ES kernel (nufft_execute_grad).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/nufft_serve.h"
#include "nufft_internal.cuh"

using namespace nufft;

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ------------------------------------------------------------------ kernels
template <typename T>
struct C2 {
  T re, im;
};

// r2_j = 2 (c_j - y_j); loss += sum_j |c_j - y_j|^2 (block sums, one double atomic per block)
template <typename T>
__global__ void k_lsq_residual(int64_t M, const C2<T>* __restrict__ c, const C2<T>* __restrict__ y,
                               C2<T>* __restrict__ r2, double* __restrict__ loss) {
  double acc = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M; j += (int64_t)gridDim.x * blockDim.x) {
    C2<T> a = c[j], b = y[j];
    T dr = a.re - b.re, di = a.im - b.im;
    r2[j] = C2<T>{dr + dr, di + di};
    acc += (double)dr * (double)dr + (double)di * (double)di;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double part[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) part[wid] = acc;
  __syncthreads();
  if (wid == 0) {
    acc = lane < (int)(blockDim.x >> 5) ? part[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) atomicAdd(loss, acc);
  }
}

// out_k = (s i k_d) f_k on the mode array (dimension 1 fastest, increasing k)
template <typename T>
__global__ void k_mul_ik(int64_t ntot, int64_t N0, int64_t N1, int64_t N2, int d, int s,
                         const C2<T>* __restrict__ f, C2<T>* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ntot; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t pos = d == 0 ? i % N0 : (d == 1 ? (i / N0) % N1 : i / (N0 * N1));
    int64_t Nd = d == 0 ? N0 : (d == 1 ? N1 : N2);
    T k = (T)(s * (pos - Nd / 2));
    C2<T> v = f[i];
    out[i] = C2<T>{-k * v.im, k * v.re};
  }
}

// gx_j = Re(conj(r2_j) cd_j)
template <typename T>
__global__ void k_gradx(int64_t M, const C2<T>* __restrict__ r2, const C2<T>* __restrict__ cd, T* __restrict__ gx) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M; j += (int64_t)gridDim.x * blockDim.x) {
    C2<T> a = r2[j], b = cd[j];
    gx[j] = a.re * b.re + a.im * b.im;
  }
}

int grid1d(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

bool valid_shape(const nufft_request* r) {
  if (!r) return false;
  if (r->kind < NUFFT_REQ_TYPE1 || r->kind > NUFFT_REQ_LSQ_GRAD) return false;
  if (r->dim < 1 || r->dim > 3 || (r->isign != 1 && r->isign != -1)) return false;
  if (r->prec != NUFFT_C64 && r->prec != NUFFT_C128) return false;
  if (!(r->eps > 0.0) || r->M < 0 || r->M >= ((int64_t)1 << 31) - 1) return false;
  if (r->upsampfac != 0.0 && r->upsampfac != 2.0 && r->upsampfac != 1.25) return false;
  for (int i = 0; i < r->dim; ++i)
    if (r->nmodes[i] < 1 || r->nmodes[i] > (1 << 29)) return false;
  return true;
}

bool valid_request(const nufft_request* r) {
  if (!valid_shape(r)) return false;
  if (!r->in || !r->out) return false;
  if (r->M > 0 && (!r->x || (r->dim > 1 && !r->y) || (r->dim > 2 && !r->z))) return false;
  if (r->kind == NUFFT_REQ_LSQ_GRAD && (!r->out3 || (r->M > 0 && (!r->in2 || !r->out2)))) return false;
  return true;
}

int64_t ntot_of(const nufft_request* r) {
  int64_t t = 1;
  for (int i = 0; i < r->dim; ++i) t *= r->nmodes[i];
  return t;
}

// point capacity of a new entry: the next power of two (at least 4096)
int64_t capacity_for(int64_t M) {
  int64_t c = 4096;
  while (c < M) c <<= 1;
  return std::min<int64_t>(c, std::max<int64_t>(M, ((int64_t)1 << 31) - 2));
}

struct Key {
  int kind, dim, isign, prec;
  int64_t n[3];
  double eps, sigma;
  bool operator==(const Key& o) const {
    return kind == o.kind && dim == o.dim && isign == o.isign && prec == o.prec && n[0] == o.n[0] &&
           n[1] == o.n[1] && n[2] == o.n[2] && eps == o.eps && sigma == o.sigma;
  }
};

Key key_of(const nufft_request* r) {
  Key k{r->kind, r->dim, r->isign, r->prec, {1, 1, 1}, r->eps, r->upsampfac};
  for (int i = 0; i < r->dim; ++i) k.n[i] = r->nmodes[i];
  return k;
}

// Upsampling factor for a request (see nufft_request_upsampfac).
double choose_sigma(const nufft_request* r) {
  if (r->upsampfac == 2.0 || r->upsampfac == 1.25) return r->upsampfac;
  int w2, w5;
  double b;
  int64_t n2[3] = {1, 1, 1}, n5[3] = {1, 1, 1};
  if (nufft_choose_params_sigma(r->dim, r->nmodes, r->eps, r->prec, 2.0, &w2, &b, n2) < 0) return 2.0;
  if (nufft_choose_params_sigma(r->dim, r->nmodes, r->eps, r->prec, 1.25, &w5, &b, n5) != NUFFT_OK) return 2.0;
  const double a = 13e-12, bb = 0.7e-12;  // s per fine-grid cell, s per stencil cell of a point
  auto cost = [&](const int64_t* n, int w) {
    double cells = (double)n[0] * (double)n[1] * (double)n[2], sten = 1.0;
    for (int i = 0; i < r->dim; ++i) sten *= w;
    return a * cells + bb * (double)r->M * sten;
  };
  return cost(n5, w5) < cost(n2, w2) ? 1.25 : 2.0;
}

// ------------------------------------------------------------ GPU executor
struct GpuEntry {
  nufft_plan p = nullptr;
  int kind = 0;
  void* cbuf = nullptr;  // LSQ: c, then each c_d (exact route) or the dim rows of dc (kernel route)
  void* r2 = nullptr;    // LSQ: 2 (c - y)
  void* fk = nullptr;    // LSQ: (s i k_d) f
};

struct DoneCtx {
  nufft_server s;
  int64_t ticket;
};

void CUDART_CB on_done(void* data) {
  DoneCtx* d = (DoneCtx*)data;
  nufft_server_complete(d->s, d->ticket, NUFFT_OK);
  delete d;
}

struct GpuExecutor {
  int device = 0;
  std::vector<cudaStream_t> streams;
  nufft_server server = nullptr;

  static size_t scratch_bytes(const nufft_request* r, int64_t mcap) {
    if (r->kind != NUFFT_REQ_LSQ_GRAD) return 0;
    size_t cs = r->prec == NUFFT_C128 ? 16 : 8;
    return ((2 + (size_t)r->dim) * (size_t)mcap + (size_t)ntot_of(r)) * cs;
  }

  static int estimate(void*, const nufft_request* r, int64_t mcap, size_t* bytes) {
    size_t b = 0;
    int st = plan_estimate_bytes(r->dim, r->nmodes, r->eps, r->prec, mcap, &b, r->upsampfac == 1.25 ? 1.25 : 2.0);
    if (st < 0) return st;
    *bytes = b + scratch_bytes(r, mcap);
    return NUFFT_OK;
  }

  static void free_entry(GpuEntry* e) {
    if (e->p) nufft_destroy(e->p);
    if (e->cbuf) cudaFree(e->cbuf);
    if (e->r2) cudaFree(e->r2);
    if (e->fk) cudaFree(e->fk);
    delete e;
  }

  static int create(void* ctx, const nufft_request* r, int64_t mcap, void** out, size_t* bytes) {
    GpuExecutor* ex = (GpuExecutor*)ctx;
    if (cudaSetDevice(ex->device) != cudaSuccess) return NUFFT_ERR_CUDA;
    GpuEntry* e = new (std::nothrow) GpuEntry();
    if (!e) return NUFFT_ERR_ALLOC;
    e->kind = r->kind;
    int type = r->kind == NUFFT_REQ_TYPE1 ? 1 : 2;
    nufft_opts o;
    nufft_default_opts(&o);
    o.upsampfac = r->upsampfac == 1.25 ? 1.25 : 2.0;
    int st = nufft_makeplan(type, r->dim, r->nmodes, r->isign, 1, r->eps, r->prec, ex->streams[0], &o, &e->p);
    if (st < 0) {
      e->p = nullptr;
      free_entry(e);
      return st;
    }
    int rs = plan_reserve(e->p, mcap);
    if (rs != NUFFT_OK) {
      free_entry(e);
      return rs;
    }
    size_t cs = r->prec == NUFFT_C128 ? 16 : 8;
    if (r->kind == NUFFT_REQ_LSQ_GRAD) {
      if (cudaMalloc(&e->cbuf, std::max<size_t>(16, (1 + (size_t)r->dim) * (size_t)mcap * cs)) != cudaSuccess ||
          cudaMalloc(&e->r2, std::max<size_t>(16, (size_t)mcap * cs)) != cudaSuccess ||
          cudaMalloc(&e->fk, (size_t)ntot_of(r) * cs) != cudaSuccess) {
        free_entry(e);
        return NUFFT_ERR_ALLOC;
      }
    }
    *bytes = plan_device_bytes(e->p) + scratch_bytes(r, mcap);
    *out = e;
    return NUFFT_OK;
  }

  template <typename T>
  static int run_lsq(GpuEntry* e, const nufft_request* r, cudaStream_t st) {
    const int s = r->isign;
    const int64_t M = r->M;
    const int64_t ntot = ntot_of(r);
    const bool kern = (r->flags & NUFFT_FLAG_XGRAD_KERNEL) != 0;
    C2<T>* dcb = (C2<T>*)e->cbuf + M;  // kernel route: dc rows after c
    int rc = kern ? plan_execute_grad(e->p, e->cbuf, dcb, r->in) : plan_execute_as(e->p, 2, s, e->cbuf, (void*)r->in);
    if (rc != NUFFT_OK) return rc;
    if (cudaMemsetAsync(r->out3, 0, sizeof(double), st) != cudaSuccess) return NUFFT_ERR_CUDA;
    if (M > 0) {
      k_lsq_residual<T><<<grid1d(M), 256, 0, st>>>(M, (const C2<T>*)e->cbuf, (const C2<T>*)r->in2, (C2<T>*)e->r2,
                                                    (double*)r->out3);
      if (cudaGetLastError() != cudaSuccess) return NUFFT_ERR_CUDA;
    }
    rc = plan_execute_as(e->p, 1, -s, e->r2, r->out);
    if (rc != NUFFT_OK) return rc;
    if (M == 0) return NUFFT_OK;
    if (kern) {
      for (int d = 0; d < r->dim; ++d) {
        k_gradx<T><<<grid1d(M), 256, 0, st>>>(M, (const C2<T>*)e->r2, dcb + d * M, (T*)r->out2 + d * M);
        if (cudaGetLastError() != cudaSuccess) return NUFFT_ERR_CUDA;
      }
      return NUFFT_OK;
    }
    int64_t N[3] = {1, 1, 1};
    for (int i = 0; i < r->dim; ++i) N[i] = r->nmodes[i];
    for (int d = 0; d < r->dim; ++d) {
      k_mul_ik<T><<<grid1d(ntot), 256, 0, st>>>(ntot, N[0], N[1], N[2], d, s, (const C2<T>*)r->in, (C2<T>*)e->fk);
      if (cudaGetLastError() != cudaSuccess) return NUFFT_ERR_CUDA;
      rc = plan_execute_as(e->p, 2, s, e->cbuf, e->fk);
      if (rc != NUFFT_OK) return rc;
      k_gradx<T><<<grid1d(M), 256, 0, st>>>(M, (const C2<T>*)e->r2, (const C2<T>*)e->cbuf, (T*)r->out2 + d * M);
      if (cudaGetLastError() != cudaSuccess) return NUFFT_ERR_CUDA;
    }
    return NUFFT_OK;
  }

  static int launch(void* ctx, void* entry, const nufft_request* r, int slot, int skip_binning, int64_t ticket) {
    GpuExecutor* ex = (GpuExecutor*)ctx;
    GpuEntry* e = (GpuEntry*)entry;
    if (cudaSetDevice(ex->device) != cudaSuccess) return NUFFT_ERR_CUDA;
    cudaStream_t st = ex->streams[slot];
    int rc = plan_set_stream(e->p, st);
    if (rc == NUFFT_OK && r->ready_event && cudaStreamWaitEvent(st, (cudaEvent_t)r->ready_event, 0) != cudaSuccess)
      rc = NUFFT_ERR_CUDA;
    if (rc == NUFFT_OK && !skip_binning) rc = nufft_setpts(e->p, r->M, r->x, r->y, r->z);
    if (rc == NUFFT_OK) {
      if (r->kind == NUFFT_REQ_TYPE1) rc = nufft_execute(e->p, (void*)r->in, r->out);
      else if (r->kind == NUFFT_REQ_TYPE2) rc = nufft_execute(e->p, r->out, (void*)r->in);
      else rc = r->prec == NUFFT_C128 ? run_lsq<double>(e, r, st) : run_lsq<float>(e, r, st);
    }
    if (rc == NUFFT_OK) {
      DoneCtx* d = new (std::nothrow) DoneCtx{ex->server, ticket};
      if (!d) rc = NUFFT_ERR_ALLOC;
      else if (cudaLaunchHostFunc(st, on_done, d) != cudaSuccess) {
        delete d;
        rc = NUFFT_ERR_CUDA;
      }
    }
    // on failure, let what was enqueued finish before the entry is handed out again
    if (rc != NUFFT_OK) cudaStreamSynchronize(st);
    return rc;
  }

  static void destroy(void* ctx, void* entry) {
    GpuExecutor* ex = (GpuExecutor*)ctx;
    cudaSetDevice(ex->device);
    free_entry((GpuEntry*)entry);
  }
};

}  // namespace

// ----------------------------------------------------------------- scheduler
struct nufft_server_s {
  nufft_executor ex{};
  GpuExecutor* gpu = nullptr;  // owned when the server runs on the GPU
  size_t budget = 0;
  int max_inflight = 1;
  double timeout = 0;
  double shutdown_wait = 60.0;  // destroy: how long to wait for running work

  struct Entry {
    void* h = nullptr;
    Key key{};
    int64_t mcap = 0;
    size_t bytes = 0;
    bool busy = false;
    uint64_t last_use = 0;
    uint64_t pkey = 0;  // points resident in the entry (0: none known)
    int64_t pM = -1;
  };
  struct Req {
    nufft_request r{};
    int64_t ticket = 0;
    double t_submit = 0, t_admit = 0;
    Entry* e = nullptr;
    int slot = -1;
    int reused = 0;
    bool reported = false;  // completion already handed to the client (time limit)
  };
  struct Fin {
    int64_t ticket;
    int status;
    double t;
  };

  // shared with client threads and completion callbacks (under mu)
  std::mutex mu;
  std::condition_variable cv_worker, cv_client;
  std::deque<Req*> queue;
  std::vector<Fin> finished;
  std::deque<nufft_completion> done;
  uint64_t events = 0;
  bool stop = false;
  int64_t next_ticket = 1;
  int64_t n_inflight = 0;
  nufft_server_stats st{};

  // scheduler thread only
  std::vector<Entry*> entries;
  std::unordered_map<int64_t, Req*> inflight;
  std::vector<int> free_slots;
  size_t used = 0;
  uint64_t use_clock = 0;
  std::thread worker;

  void report(std::vector<nufft_completion>& out, Req* q, int status, double t, int pending = 0) {
    nufft_completion c;
    c.ticket = q->ticket;
    c.tag = q->r.tag;
    c.status = status;
    c.reused = q->reused;
    c.t_submit = q->t_submit;
    c.t_admit = q->t_admit;
    c.t_done = t;
    c.pending = pending;
    out.push_back(c);
  }

  void publish(std::vector<nufft_completion>& out) {
    if (out.empty()) return;
    std::lock_guard<std::mutex> lk(mu);
    for (auto& c : out) {
      done.push_back(c);
      if (c.pending) st.timeouts++;
      else st.completed++;
      if (c.status == NUFFT_ERR_REJECTED) st.rejected++;
    }
    out.clear();
    cv_client.notify_all();
  }

  void release(Req* q) {
    if (q->e) {
      q->e->busy = false;
      q->e->last_use = ++use_clock;
    }
    if (q->slot >= 0) free_slots.push_back(q->slot);
  }

  void destroy_entry(size_t i) {
    Entry* e = entries[i];
    ex.destroy(ex.ctx, e->h);
    used -= e->bytes;
    entries.erase(entries.begin() + (long)i);
    delete e;
  }

  // best idle entry for q: same key, capacity >= M; resident points first, then the smallest capacity
  Entry* find_idle(const Req* q, bool* same_points) {
    Key k = key_of(&q->r);
    Entry* best = nullptr;
    *same_points = false;
    for (Entry* e : entries) {
      if (e->busy || !(e->key == k) || e->mcap < q->r.M) continue;
      bool sp = q->r.points_key != 0 && e->pkey == q->r.points_key && e->pM == q->r.M;
      if (sp && !*same_points) {
        best = e;
        *same_points = true;
      } else if (!*same_points && (!best || e->mcap < best->mcap)) {
        best = e;
      }
    }
    return best;
  }

  // 1: admitted or finished (rejected / failed); 0: must wait for running work
  int try_admit(Req* q, std::vector<nufft_completion>& out) {
    bool same = false;
    Entry* e = find_idle(q, &same);
    int reused = e ? (same ? 2 : 1) : 0;
    if (!e) {
      const int64_t mcap = capacity_for(q->r.M);
      size_t need = 0;
      int rc = ex.estimate(ex.ctx, &q->r, mcap, &need);
      if (rc < 0) {
        report(out, q, rc, now_s());
        return 1;
      }
      if (need > budget) {
        report(out, q, NUFFT_ERR_REJECTED, now_s());
        return 1;
      }
      size_t idle = 0;
      for (Entry* x : entries)
        if (!x->busy) idle += x->bytes;
      if (used - idle + need > budget) return 0;  // only running work can free enough
      while (used + need > budget) {              // evict idle entries, least recently used first
        size_t lru = entries.size();
        for (size_t i = 0; i < entries.size(); ++i)
          if (!entries[i]->busy && (lru == entries.size() || entries[i]->last_use < entries[lru]->last_use))
            lru = i;
        destroy_entry(lru);
        std::lock_guard<std::mutex> lk(mu);
        st.entries_evicted++;
      }
      void* h = nullptr;
      size_t bytes = 0;
      rc = ex.create(ex.ctx, &q->r, mcap, &h, &bytes);
      if (rc < 0) {
        report(out, q, rc, now_s());
        return 1;
      }
      e = new Entry();
      e->h = h;
      e->key = key_of(&q->r);
      e->mcap = mcap;
      e->bytes = bytes;
      entries.push_back(e);
      used += bytes;
      std::lock_guard<std::mutex> lk(mu);
      st.entries_created++;
    }
    const int slot = free_slots.back();
    free_slots.pop_back();
    e->busy = true;
    q->e = e;
    q->slot = slot;
    q->reused = reused;
    q->t_admit = now_s();
    int rc = ex.launch(ex.ctx, e->h, &q->r, slot, same ? 1 : 0, q->ticket);
    if (rc < 0) {
      e->pkey = 0;
      e->pM = -1;
      release(q);
      report(out, q, rc, now_s());
      return 1;
    }
    e->pkey = q->r.points_key;
    e->pM = q->r.M;
    inflight[q->ticket] = q;
    std::lock_guard<std::mutex> lk(mu);
    n_inflight++;
    st.inflight = n_inflight;
    st.peak_inflight = std::max(st.peak_inflight, n_inflight);
    if (reused) st.entries_reused++;
    if (same) st.binning_skipped++;
    st.bytes_in_use = (int64_t)used;
    st.peak_bytes = std::max(st.peak_bytes, (int64_t)used);
    return 1;
  }

  // the request's work has ended: its final completion (a second one after an early time-limit report)
  void retire(Req* q, std::vector<nufft_completion>& out, int status, double t) {
    report(out, q, status, t);
    release(q);
    inflight.erase(q->ticket);
    delete q;
    std::lock_guard<std::mutex> lk(mu);
    n_inflight--;
    st.inflight = n_inflight;
    st.bytes_in_use = (int64_t)used;
    cv_client.notify_all();
  }

  void run() {
    std::vector<nufft_completion> out;
    for (;;) {
      std::vector<Fin> fin;
      uint64_t seen;
      bool stopping;
      {
        std::lock_guard<std::mutex> lk(mu);
        fin.swap(finished);
        seen = events;
        stopping = stop;
      }
      for (const Fin& f : fin) {
        auto it = inflight.find(f.ticket);
        if (it != inflight.end()) retire(it->second, out, f.status, f.t);
      }
      if (timeout > 0) {
        const double t = now_s();
        for (auto& kv : inflight) {
          Req* q = kv.second;
          if (!q->reported && t >= q->t_admit + timeout) {
            report(out, q, NUFFT_ERR_TIMEOUT, t, 1);  // early: the work is still running
            q->reported = true;
          }
        }
      }
      if (stopping) break;
      while (!free_slots.empty()) {
        Req* q;
        {
          std::lock_guard<std::mutex> lk(mu);
          if (queue.empty()) break;
          q = queue.front();
        }
        if (!try_admit(q, out)) break;
        std::lock_guard<std::mutex> lk(mu);
        queue.pop_front();
        st.queued = (int64_t)queue.size();
        cv_client.notify_all();
        if (!inflight.count(q->ticket)) delete q;  // finished without running
      }
      publish(out);
      double next_deadline = 0;  // earliest time limit among running requests
      if (timeout > 0)
        for (auto& kv : inflight)
          if (!kv.second->reported) {
            double dl = kv.second->t_admit + timeout;
            if (next_deadline == 0 || dl < next_deadline) next_deadline = dl;
          }
      std::unique_lock<std::mutex> lk(mu);
      auto ready = [&] { return events != seen || stop; };
      if (next_deadline > 0) {
        auto wait = std::chrono::duration<double>(std::max(0.0, next_deadline - now_s()));
        cv_worker.wait_for(lk, wait, ready);
      } else {
        cv_worker.wait(lk, ready);
      }
    }
    // shutting down: fail what is queued, let running work finish, free the entries
    {
      std::lock_guard<std::mutex> lk(mu);
      for (Req* q : queue) {
        nufft_completion c{q->ticket, q->r.tag, NUFFT_ERR_SHUTDOWN, 0, q->t_submit, 0.0, now_s(), 0};
        done.push_back(c);
        st.completed++;
        delete q;
      }
      queue.clear();
      st.queued = 0;
    }
    if (gpu)
      for (cudaStream_t s : gpu->streams) cudaStreamSynchronize(s);
    double wait_s;
    {
      std::lock_guard<std::mutex> lk(mu);
      wait_s = shutdown_wait;
    }
    const double give_up = now_s() + wait_s;
    while (!inflight.empty() && now_s() < give_up) {
      std::vector<Fin> fin;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_worker.wait_for(lk, std::chrono::milliseconds(10), [&] { return !finished.empty(); });
        fin.swap(finished);
      }
      for (const Fin& f : fin) {
        auto it = inflight.find(f.ticket);
        if (it != inflight.end()) retire(it->second, out, f.status, f.t);
      }
      publish(out);
    }
    // the executor never reported these requests: their entries may still be in use on the device, so
    // they are leaked (not destroyed); the requests themselves get no final completion
    for (auto& kv : inflight) delete kv.second;
    inflight.clear();
    while (!entries.empty()) {
      Entry* e = entries.back();
      if (e->busy) {
        used -= e->bytes;
        entries.pop_back();
        delete e;
      } else {
        destroy_entry(entries.size() - 1);
      }
    }
    publish(out);
  }
};

namespace {

int server_start(nufft_server s, size_t budget, int max_inflight, double timeout_s) {
  s->budget = budget;
  s->max_inflight = max_inflight;
  s->timeout = timeout_s > 0 ? timeout_s : 0;
  s->st.budget_bytes = (int64_t)budget;
  for (int i = max_inflight - 1; i >= 0; --i) s->free_slots.push_back(i);
  try {
    s->worker = std::thread([s] { s->run(); });
  } catch (...) {
    return NUFFT_ERR_ALLOC;
  }
  return NUFFT_OK;
}

}  // namespace

extern "C" {

double nufft_server_clock(void) { return now_s(); }

double nufft_request_upsampfac(const nufft_request* r) { return valid_shape(r) ? choose_sigma(r) : 0.0; }

int nufft_request_bytes(const nufft_request* r, int64_t mcap, size_t* bytes) {
  if (!valid_shape(r) || !bytes || mcap < r->M) return NUFFT_ERR_BAD_ARG;
  nufft_request q = *r;
  q.upsampfac = choose_sigma(r);
  return GpuExecutor::estimate(nullptr, &q, mcap, bytes);
}

int nufft_server_create(size_t budget_bytes, int max_inflight, double timeout_s, nufft_server* out) {
  if (!out || max_inflight < 1 || max_inflight > 64 || budget_bytes == 0) return NUFFT_ERR_BAD_ARG;
  *out = nullptr;
  nufft_server s = new (std::nothrow) nufft_server_s();
  if (!s) return NUFFT_ERR_ALLOC;
  GpuExecutor* g = new (std::nothrow) GpuExecutor();
  if (!g) {
    delete s;
    return NUFFT_ERR_ALLOC;
  }
  g->server = s;
  bool ok = cudaGetDevice(&g->device) == cudaSuccess;
  for (int i = 0; ok && i < max_inflight; ++i) {
    cudaStream_t st;
    ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) g->streams.push_back(st);
  }
  if (!ok) {
    for (cudaStream_t st : g->streams) cudaStreamDestroy(st);
    delete g;
    delete s;
    return NUFFT_ERR_CUDA;
  }
  s->gpu = g;
  s->ex.ctx = g;
  s->ex.estimate = &GpuExecutor::estimate;
  s->ex.create = &GpuExecutor::create;
  s->ex.launch = &GpuExecutor::launch;
  s->ex.destroy = &GpuExecutor::destroy;
  int rc = server_start(s, budget_bytes, max_inflight, timeout_s);
  if (rc != NUFFT_OK) {
    for (cudaStream_t st : g->streams) cudaStreamDestroy(st);
    delete g;
    delete s;
    return rc;
  }
  *out = s;
  return NUFFT_OK;
}

int nufft_server_create_with_executor(const nufft_executor* ex, size_t budget_bytes, int max_inflight,
                                      double timeout_s, nufft_server* out) {
  if (!out || !ex || !ex->estimate || !ex->create || !ex->launch || !ex->destroy || max_inflight < 1 ||
      max_inflight > 64 || budget_bytes == 0)
    return NUFFT_ERR_BAD_ARG;
  *out = nullptr;
  nufft_server s = new (std::nothrow) nufft_server_s();
  if (!s) return NUFFT_ERR_ALLOC;
  s->ex = *ex;
  int rc = server_start(s, budget_bytes, max_inflight, timeout_s);
  if (rc != NUFFT_OK) {
    delete s;
    return rc;
  }
  *out = s;
  return NUFFT_OK;
}

int nufft_server_submit(nufft_server s, const nufft_request* r, int64_t* ticket) {
  if (!s || !valid_request(r)) return NUFFT_ERR_BAD_ARG;
  nufft_server_s::Req* q = new (std::nothrow) nufft_server_s::Req();
  if (!q) return NUFFT_ERR_ALLOC;
  q->r = *r;
  q->r.upsampfac = choose_sigma(r);  // resolved once: the key, the estimate and the plan all use it
  q->t_submit = now_s();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) {
    delete q;
    return NUFFT_ERR_SHUTDOWN;
  }
  q->ticket = s->next_ticket++;
  if (ticket) *ticket = q->ticket;
  s->queue.push_back(q);
  s->st.submitted++;
  s->st.queued = (int64_t)s->queue.size();
  s->events++;
  s->cv_worker.notify_one();
  return NUFFT_OK;
}

int nufft_server_set_shutdown_wait(nufft_server s, double seconds) {
  if (!s || !(seconds > 0)) return NUFFT_ERR_BAD_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  s->shutdown_wait = seconds;
  return NUFFT_OK;
}

void nufft_server_complete(nufft_server s, int64_t ticket, int status) {
  if (!s) return;
  const double t = now_s();
  std::lock_guard<std::mutex> lk(s->mu);
  s->finished.push_back({ticket, status, t});
  s->events++;
  s->cv_worker.notify_one();
}

int nufft_server_poll(nufft_server s, nufft_completion* out, int max, int* n, double wait_s) {
  if (!s || !n || max < 0 || (max > 0 && !out)) return NUFFT_ERR_BAD_ARG;
  *n = 0;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && wait_s > 0)
    s->cv_client.wait_for(lk, std::chrono::duration<double>(wait_s), [&] { return !s->done.empty(); });
  int k = 0;
  while (k < max && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  *n = k;
  return NUFFT_OK;
}

int nufft_server_drain(nufft_server s, double timeout_s) {
  if (!s) return NUFFT_ERR_BAD_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto idle = [&] { return s->queue.empty() && s->n_inflight == 0; };
  if (timeout_s > 0) {
    if (!s->cv_client.wait_for(lk, std::chrono::duration<double>(timeout_s), idle)) return NUFFT_ERR_TIMEOUT;
  } else {
    s->cv_client.wait(lk, idle);
  }
  return NUFFT_OK;
}

int nufft_server_stats_get(nufft_server s, nufft_server_stats* st) {
  if (!s || !st) return NUFFT_ERR_BAD_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *st = s->st;
  return NUFFT_OK;
}

int nufft_server_destroy(nufft_server s) {
  if (!s) return NUFFT_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->events++;
    s->cv_worker.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  if (s->gpu) {
    cudaSetDevice(s->gpu->device);
    for (cudaStream_t st : s->gpu->streams) cudaStreamDestroy(st);
    delete s->gpu;
  }
  delete s;
  return NUFFT_OK;
}

}  // extern "C"
