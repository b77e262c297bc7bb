// serve.cu -- continuous-batching server of independent solves (sem.h,
// "Serving").  The paper solves one large problem at a time; the server runs
// streams of independent problems (many small and mid-sized boxes) so that
// their kernels overlap on one GPU.
//
// Structure: a FIFO of requests, `workers` host threads with one CUDA stream
// each, and a cache of idle setups (mesh + pMG hierarchy) keyed by the mesh
// shape.  A worker takes the head of the queue when its estimated device
// memory fits in the budget (or when nothing else is running), reuses or
// builds a setup, solves through the library's own ABI on its stream, copies x
// back and records the result.  Admission is by device bytes measured on
// earlier setups: the exact bytes of a shape built before, else the largest
// bytes per local point measured for the request's order, else (before any
// setup of that order) a first estimate; once a new setup has solved, its
// reservation is replaced by what it holds.  The budget counts running and
// cached setups, and idle cached setups of other shapes are released to make
// room.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <system_error>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "pmg.cuh"

namespace sem {

// b_l = B_l f(x_l), f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z): the manufactured
// right-hand side of -lap u = f with u = sin sin sin (gs and mask follow).
__global__ void manufactured_rhs_kernel(int64_t n, const double *__restrict__ X,
                                        const double *__restrict__ Y,
                                        const double *__restrict__ Z,
                                        const double *__restrict__ B, double *__restrict__ b) {
  const double pi = 3.14159265358979323846;
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
       l += (int64_t)gridDim.x * blockDim.x)
    b[l] = B[l] * 3.0 * pi * pi * sin(pi * X[l]) * sin(pi * Y[l]) * sin(pi * Z[l]);
}

void build_manufactured_rhs(const Level &L, double *b, double *tmp, cudaStream_t st) {
  const int64_t nl = L.t.nl;
  double *X = tmp, *Y = X + nl, *Z = Y + nl, *B = Z + nl;
  launch_field(L, SEM_FIELD_X, X, st);
  launch_field(L, SEM_FIELD_Y, Y, st);
  launch_field(L, SEM_FIELD_Z, Z, st);
  launch_field(L, SEM_FIELD_MASS, B, st);
  manufactured_rhs_kernel<<<vec_grid(nl), kVecThreads, 0, st>>>(nl, X, Y, Z, B, b);
  SEM_CHECK_CUDA(cudaGetLastError());
  launch_gs<double>(L, b, st);
  launch_mask<double>(L, b, st);
}

namespace {

using Clock = std::chrono::steady_clock;

struct ShapeKey {
  int32_t ex, ey, ez, N, bc;
  double jitter;
  uint64_t seed;
  bool operator<(const ShapeKey &o) const {
    return std::tie(ex, ey, ez, N, bc, jitter, seed) <
           std::tie(o.ex, o.ey, o.ez, o.N, o.bc, o.jitter, o.seed);
  }
};

struct Setup {
  ShapeKey key{};
  sem_mesh *mesh = nullptr;
  sem_pmg *pmg = nullptr;
  DevBuf<double> b, x, tmp;
  int64_t bytes = 0;
  ~Setup() {
    if (pmg) sem_pmg_destroy(pmg);
    if (mesh) sem_mesh_destroy(mesh);
  }
};

struct Request {
  sem_request r{};
  ShapeKey key{};
  std::vector<double> b;  // host copy of the right-hand side
  int64_t est_bytes = 0;
  Clock::time_point submitted;
  int state = 0;  // 0 queued, 1 running, 2 done
  sem_status status = SEM_OK;
  sem_solve_info info{};
};

int64_t local_points(const ShapeKey &k) {
  return (int64_t)k.ex * k.ey * k.ez * (k.N + 1) * (k.N + 1) * (k.N + 1);
}

// A first guess of one setup's device bytes, used only until a setup of the
// same order has been measured: 200 bytes per local point (FP64 operator
// factors and work vectors, the FP32 smoothing levels, the coarse solver)
// plus a fixed part.
int64_t estimate_bytes(const ShapeKey &k) { return 200 * local_points(k) + (64ll << 20); }

std::vector<int32_t> level_orders(int N) {
  std::vector<int32_t> o{N};
  const int c = N / 2;
  if (c > 1 && c < N) o.push_back(c);
  if (N > 1) o.push_back(1);
  return o;
}

}  // namespace
}  // namespace sem

using namespace sem;

struct sem_server {
  sem_server_desc d{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  std::multimap<ShapeKey, std::unique_ptr<Setup>> cache;  // idle setups
  std::deque<Setup *> cache_lru;                          // oldest first
  int64_t in_use = 0;
  // measured device bytes: of every shape built so far, and the largest
  // bytes per local point seen per order (admission of unseen shapes)
  std::map<ShapeKey, int64_t> measured;
  std::map<int, double> rate_by_order;
  int64_t admit_bytes_locked(const ShapeKey &k) const {
    auto m = measured.find(k);
    if (m != measured.end()) return m->second;
    auto r = rate_by_order.find(k.N);
    if (r != rate_by_order.end()) return (int64_t)std::ceil(1.05 * r->second * local_points(k));
    return estimate_bytes(k);
  }
  int running = 0;
  bool stop = false;
  uint64_t next_ticket = 1;
  sem_server_stats stats{};
  std::vector<std::thread> threads;

  void worker();
  std::unique_ptr<Setup> build(const ShapeKey &k, cudaStream_t st);
  void serve_one(Request &q, Setup &S, cudaStream_t st);
  bool evict_one_locked(const ShapeKey *keep);
};

bool sem_server::evict_one_locked(const ShapeKey *keep) {
  for (auto it = cache_lru.begin(); it != cache_lru.end(); ++it) {
    Setup *s = *it;
    if (keep && !(s->key < *keep) && !(*keep < s->key)) continue;
    auto range = cache.equal_range(s->key);
    for (auto c = range.first; c != range.second; ++c) {
      if (c->second.get() == s) {
        in_use -= s->bytes;
        cache_lru.erase(it);
        cache.erase(c);  // frees the setup
        return true;
      }
    }
  }
  return false;
}

std::unique_ptr<Setup> sem_server::build(const ShapeKey &k, cudaStream_t st) {
  std::unique_ptr<Setup> S(new Setup());
  S->key = k;
  sem_mesh_desc md{};
  md.ex = k.ex;
  md.ey = k.ey;
  md.ez = k.ez;
  md.N = k.N;
  md.jitter = k.jitter;
  md.seed = k.seed;
  md.bc = k.bc;
  md.geom = SEM_GEOM_STORED;
  md.verts = nullptr;
  md.f64_arith = SEM_ARITH_PAIR;
  sem_status s = sem_mesh_create(&md, st, &S->mesh);
  if (s != SEM_OK) fail(s, "server: mesh creation failed: %s", sem_last_error());
  const std::vector<int32_t> ord = level_orders(k.N);
  sem_pmg_desc pd{};
  pd.nlevels = (int32_t)ord.size();
  for (size_t i = 0; i < ord.size(); ++i) pd.orders[i] = ord[i];
  pd.cheb_degree = d.cheb_degree;
  pd.lanczos_steps = 20;
  pd.seed = 0;
  pd.smoother_dtype = d.smoother_dtype;
  pd.coarse_tol = d.coarse_tol;
  pd.coarse_maxit = d.coarse_maxit;
  pd.coarse_mode = SEM_COARSE_MG;
  s = sem_pmg_setup(S->mesh, &pd, st, &S->pmg);
  if (s != SEM_OK) fail(s, "server: pMG setup failed: %s", sem_last_error());
  const int64_t nl = S->mesh->fine.t.nl;
  S->b.alloc(nl);
  S->x.alloc(nl);
  S->bytes = 0;  // measured after its first solve (setup_bytes)
  return S;
}

// Device bytes a setup holds: mesh (with its solver workspaces), hierarchy,
// right-hand side, solution and scratch.
static int64_t setup_bytes(const Setup &S) {
  size_t mb = 0;
  sem_mesh_info(S.mesh, nullptr, nullptr, &mb);
  return (int64_t)(mb + pmg_device_bytes(S.pmg) + S.b.bytes() + S.x.bytes() + S.tmp.bytes());
}

void sem_server::serve_one(Request &q, Setup &S, cudaStream_t st) {
  const Level &L = S.mesh->fine;
  const int64_t nl = L.t.nl;
  if (q.r.rhs == SEM_RHS_MANUFACTURED) {
    if (!S.tmp.p) S.tmp.alloc(4 * (size_t)nl);
    build_manufactured_rhs(L, S.b.p, S.tmp.p, st);
  } else {
    SEM_CHECK_CUDA(cudaMemcpyAsync(S.b.p, q.b.data(), nl * sizeof(double),
                                   cudaMemcpyHostToDevice, st));
  }
  // requests start from x = 0 (their x is output only)
  sem_solve_desc sd = q.r.solve;
  sd.zero_guess = 1;
  sem_solve_info info{};
  const sem_status s = sem_solve(S.mesh, S.pmg, S.b.p, S.x.p, &sd, &info, st);
  if (s != SEM_OK && s != SEM_ENOTCONV) fail(s, "server: solve failed: %s", sem_last_error());
  if (q.r.x)
    SEM_CHECK_CUDA(cudaMemcpyAsync(q.r.x, S.x.p, nl * sizeof(double), cudaMemcpyDeviceToHost, st));
  SEM_CHECK_CUDA(cudaStreamSynchronize(st));
  q.info = info;
  q.status = s;
}

void sem_server::worker() {
  cudaSetDevice(device);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
  for (;;) {
    std::unique_ptr<Setup> S;
    Request *q = nullptr;
    {
      std::unique_lock<std::mutex> lk(mu);
      for (;;) {
        if (!queue.empty()) {
          Request &h = *reqs[queue.front()];
          auto hit = cache.find(h.key);
          if (hit != cache.end()) {  // reuse an idle setup of this shape
            S = std::move(hit->second);
            cache_lru.erase(std::find(cache_lru.begin(), cache_lru.end(), S.get()));
            cache.erase(hit);
            stats.setups_reused += 1;
            q = &h;
            break;
          }
          h.est_bytes = admit_bytes_locked(h.key);
          while (in_use + h.est_bytes > d.hbm_budget && evict_one_locked(nullptr)) {
          }
          if (in_use + h.est_bytes <= d.hbm_budget || running == 0) {
            in_use += h.est_bytes;
            q = &h;
            break;
          }
        } else if (stop) {
          break;
        }
        cv_work.wait(lk);
      }
      if (!q) break;
      queue.pop_front();
      q->state = 1;
      running += 1;
    }
    sem_status status = SEM_OK;
    const bool built = !S;
    try {
      if (!S) S = build(q->key, st);
      serve_one(*q, *S, st);
      if (built) {
        // replace the admission's reservation by what the setup holds
        const int64_t b = setup_bytes(*S);
        std::lock_guard<std::mutex> lk(mu);
        in_use += b - q->est_bytes;
        S->bytes = b;
        measured[q->key] = b;
        const double rate = (double)b / (double)local_points(q->key);
        double &r = rate_by_order[q->key.N];
        r = std::max(r, rate);
      }
    } catch (const Failure &f) {
      status = f.status;
      if (st) cudaStreamSynchronize(st);
    } catch (...) {
      status = SEM_ECUDA;
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      if (status != SEM_OK) q->status = status;
      q->info.status = q->status;
      q->info.time_ms =
          std::chrono::duration<double, std::milli>(Clock::now() - q->submitted).count();
      q->state = 2;
      running -= 1;
      stats.completed += 1;
      if (q->status != SEM_OK) stats.failed += 1;
      if (built && S) stats.setups_built += 1;
      if (built && S && S->bytes == 0) S->bytes = q->est_bytes;  // failed before measuring
      if (built && !S) in_use -= q->est_bytes;  // the build failed: nothing is held
      if (S) {
        const size_t kept = cache.count(S->key);
        if (status == SEM_OK && (int)kept < d.cache_per_shape) {
          cache_lru.push_back(S.get());
          cache.emplace(S->key, std::move(S));
        } else {
          in_use -= S->bytes;
          S.reset();
        }
      }
    }
    cv_done.notify_all();
    cv_work.notify_all();
  }
  if (st) cudaStreamDestroy(st);
}

namespace {

template <typename F>
sem_status serve_guard(F &&f) {
  try {
    f();
    return SEM_OK;
  } catch (const Failure &e) {
    return e.status;
  } catch (const std::bad_alloc &) {
    set_error_message("host allocation failed");
    return SEM_ENOMEM;
  } catch (const std::system_error &) {
    set_error_message("could not start a server thread");
    return SEM_ENOMEM;
  } catch (...) {
    set_error_message("unexpected internal error");
    return SEM_ECUDA;
  }
}

void check_desc(const sem_server_desc *d) {
  SEM_REQUIRE(d != nullptr, "null server description");
  SEM_REQUIRE(d->workers >= 1 && d->workers <= 64, "workers %d outside [1, 64]", d->workers);
  SEM_REQUIRE(d->hbm_budget >= 0 && d->cache_per_shape >= 0, "negative budget or cache size");
  SEM_REQUIRE(d->cheb_degree >= 1 && d->cheb_degree <= 16, "cheb_degree outside [1, 16]");
  SEM_REQUIRE(d->smoother_dtype >= SEM_F64 && d->smoother_dtype <= SEM_BF16, "bad smoother_dtype");
  SEM_REQUIRE(d->coarse_maxit >= 0, "negative coarse_maxit");
}

void check_request(const sem_request *r) {
  SEM_REQUIRE(r != nullptr, "null request");
  SEM_REQUIRE(r->ex >= 1 && r->ey >= 1 && r->ez >= 1, "element counts must be >= 1");
  SEM_REQUIRE((int64_t)r->ex * r->ey * r->ez <= (1ll << 31), "too many elements");
  SEM_REQUIRE(r->N >= 1 && r->N <= SEM_MAX_ORDER, "order N=%d outside [1, %d]", r->N,
              SEM_MAX_ORDER);
  SEM_REQUIRE(r->bc == SEM_DIRICHLET || r->bc == SEM_NEUMANN, "unknown bc %d", r->bc);
  SEM_REQUIRE(r->jitter >= 0.0 && r->jitter < 0.5, "jitter must be in [0, 0.5)");
  SEM_REQUIRE(r->rhs == SEM_RHS_HOST || r->rhs == SEM_RHS_MANUFACTURED, "unknown rhs %d", r->rhs);
  SEM_REQUIRE(r->rhs != SEM_RHS_HOST || r->b != nullptr, "SEM_RHS_HOST needs b");
  SEM_REQUIRE(r->rhs != SEM_RHS_MANUFACTURED || r->bc == SEM_DIRICHLET,
              "the manufactured right-hand side is Dirichlet");
  const sem_solve_desc &s = r->solve;
  SEM_REQUIRE(s.solver == SEM_SOLVER_PCG || s.solver == SEM_SOLVER_FLEXCG ||
                  s.solver == SEM_SOLVER_FGMRES,
              "unknown solver %d", s.solver);
  SEM_REQUIRE(s.tol >= 0.0 && s.max_iter >= 0, "negative tol or max_iter");
  SEM_REQUIRE(s.restart >= 0 && s.restart <= kMaxKrylov, "restart outside [0, %d]", kMaxKrylov);
  SEM_REQUIRE(s.use_graph == 0 || (s.use_graph == 1 && s.solver == SEM_SOLVER_FLEXCG),
              "use_graph is 0, or 1 with SEM_SOLVER_FLEXCG");
}

}  // namespace

extern "C" {

sem_status sem_server_create(const sem_server_desc *desc, sem_server **out) {
  return serve_guard([&] {
    SEM_REQUIRE(out != nullptr, "null out");
    *out = nullptr;
    check_desc(desc);
    std::unique_ptr<sem_server> S(new sem_server());
    S->d = *desc;
    SEM_CHECK_CUDA(cudaGetDevice(&S->device));
    if (S->d.hbm_budget == 0) {
      size_t fr = 0, tot = 0;
      SEM_CHECK_CUDA(cudaMemGetInfo(&fr, &tot));
      S->d.hbm_budget = (int64_t)(0.8 * (double)fr);
    }
    for (int w = 0; w < S->d.workers; ++w) S->threads.emplace_back([p = S.get()] { p->worker(); });
    *out = S.release();
  });
}

sem_status sem_server_destroy(sem_server *server) {
  return serve_guard([&] {
    if (!server) return;
    {
      std::lock_guard<std::mutex> lk(server->mu);
      server->stop = true;
    }
    server->cv_work.notify_all();
    for (auto &t : server->threads) t.join();
    server->cache_lru.clear();
    server->cache.clear();
    delete server;
  });
}

sem_status sem_submit(sem_server *server, const sem_request *req, uint64_t *ticket) {
  return serve_guard([&] {
    SEM_REQUIRE(server != nullptr && ticket != nullptr, "null server or ticket");
    check_request(req);
    std::unique_ptr<Request> q(new Request());
    q->r = *req;
    q->key = ShapeKey{req->ex, req->ey, req->ez, req->N, req->bc, req->jitter, req->seed};
    q->est_bytes = estimate_bytes(q->key);  // replaced at admission
    if (req->rhs == SEM_RHS_HOST) {
      const int64_t nl =
          (int64_t)req->ex * req->ey * req->ez * (req->N + 1) * (req->N + 1) * (req->N + 1);
      q->b.assign(req->b, req->b + nl);
    }
    q->r.b = nullptr;
    q->submitted = Clock::now();
    {
      std::lock_guard<std::mutex> lk(server->mu);
      if (server->queue.size() >= 65536) fail(SEM_EBUSY, "server queue is full");
      const uint64_t t = server->next_ticket++;
      server->reqs.emplace(t, std::move(q));
      server->queue.push_back(t);
      server->stats.submitted += 1;
      *ticket = t;
    }
    server->cv_work.notify_one();
  });
}

sem_status sem_poll(sem_server *server, uint64_t ticket, sem_solve_info *out) {
  sem_status pending = SEM_OK;
  sem_status st = serve_guard([&] {
    SEM_REQUIRE(server != nullptr && out != nullptr, "null server or out");
    std::lock_guard<std::mutex> lk(server->mu);
    auto it = server->reqs.find(ticket);
    SEM_REQUIRE(it != server->reqs.end(), "unknown ticket %llu", (unsigned long long)ticket);
    if (it->second->state != 2) {
      pending = SEM_EAGAIN;
      return;
    }
    *out = it->second->info;
    server->reqs.erase(it);
  });
  return st != SEM_OK ? st : pending;
}

sem_status sem_server_stats_read(const sem_server *server, sem_server_stats *out) {
  return serve_guard([&] {
    SEM_REQUIRE(server != nullptr && out != nullptr, "null server or out");
    sem_server *s = const_cast<sem_server *>(server);
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->hbm_in_use = s->in_use;
  });
}

sem_status sem_server_autotune(const sem_server_desc *base, const sem_request *reqs, int32_t n,
                               int32_t max_workers, int32_t *best_workers, double *best_rate) {
  return serve_guard([&] {
    SEM_REQUIRE(base && reqs && best_workers && best_rate, "null argument");
    SEM_REQUIRE(n >= 1 && max_workers >= 1 && max_workers <= 64, "bad n or max_workers");
    for (int32_t i = 0; i < n; ++i) check_request(&reqs[i]);
    *best_workers = 1;
    *best_rate = 0.0;
    for (int w = 1; w <= max_workers; w *= 2) {
      sem_server_desc d = *base;
      d.workers = w;
      sem_server *S = nullptr;
      sem_status s = sem_server_create(&d, &S);
      if (s != SEM_OK) fail(s, "autotune: %s", sem_last_error());
      std::vector<uint64_t> tickets(n);
      const auto t0 = Clock::now();
      for (int32_t i = 0; i < n; ++i) {
        s = sem_submit(S, &reqs[i], &tickets[i]);
        if (s != SEM_OK) {
          sem_server_destroy(S);
          fail(s, "autotune: %s", sem_last_error());
        }
      }
      {
        std::unique_lock<std::mutex> lk(S->mu);
        S->cv_done.wait(lk, [&] { return S->stats.completed >= S->stats.submitted; });
      }
      const double secs = std::chrono::duration<double>(Clock::now() - t0).count();
      for (int32_t i = 0; i < n; ++i) {
        sem_solve_info info{};
        sem_poll(S, tickets[i], &info);
      }
      sem_server_destroy(S);
      const double rate = n / secs;
      if (rate > *best_rate) {
        *best_rate = rate;
        *best_workers = w;
      }
    }
  });
}

}  // extern "C"
