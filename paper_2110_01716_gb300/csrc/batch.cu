// batch.cu -- many independent solves in one graph launch (sem.h, "Batched
// solves").  The paper solves one large problem at a time; a stream of small
// and mid-sized boxes leaves most of a GB300 idle when each is solved on its
// own (its kernels are short and latency-bound).  Here every problem's setup
// lives in one device arena, and one CUDA graph holds every problem's whole
// FlexCG solve from x = 0 as an independent branch: the V-cycles, operators,
// reductions and the stopping tests of all problems run on the device
// concurrently, with one launch and one read-back for the whole batch.
//
// Each branch runs exactly the kernels of sem_solve (FlexCG, zero_guess) in
// the same order, so its result equals the standalone solve on a mesh and
// pMG built from the same descriptions bit for bit.  The autotuner picks the
// FP32 operator's work split (x-line segments per resident CTA slot, i.e.
// elements per work unit and CTAs per problem) per order from timed
// launches; that split moves work between CTAs without changing any bit.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <memory>
#include <new>
#include <set>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "pmg.cuh"
#include "trace.cuh"

namespace sem {

// capi.cu
cudaGraphNode_t capture_flexcg(sem_mesh *M, sem_pmg *P, const double *b, double *x, double tol,
                               int maxit, cudaGraph_t g, cudaStream_t cs);
cudaGraphNode_t capture_slots_copy(sem_mesh *M, double *dst, cudaGraph_t g, cudaGraphNode_t after,
                                   cudaStream_t cs);
sem_status flexcg_graph_result(const double *s, sem_solve_info &info);
bool mesh_take_wait_errors(sem_mesh *M, sem_pmg *P, cudaStream_t st);
void mesh_check_rhs(sem_mesh *M, const double *b, cudaStream_t st);

namespace {

constexpr int kSlots = 16;  // result slots per problem (13 used)

std::vector<int32_t> batch_orders(int N) {
  std::vector<int32_t> o{N};
  const int c = N / 2;
  if (c > 1 && c < N) o.push_back(c);
  if (N > 1) o.push_back(1);
  return o;
}

void check_batch_request(const sem_request &r) {
  SEM_REQUIRE(r.ex >= 1 && r.ey >= 1 && r.ez >= 1, "element counts must be >= 1");
  SEM_REQUIRE((int64_t)r.ex * r.ey * r.ez <= (1ll << 31), "too many elements");
  SEM_REQUIRE(r.N >= 2 && r.N <= SEM_MAX_ORDER, "batched problems need 2 <= N <= %d (got %d)",
              SEM_MAX_ORDER, r.N);
  SEM_REQUIRE(r.bc == SEM_DIRICHLET || r.bc == SEM_NEUMANN, "unknown bc %d", r.bc);
  SEM_REQUIRE(r.jitter >= 0.0 && r.jitter < 0.5, "jitter must be in [0, 0.5)");
  SEM_REQUIRE(r.rhs == SEM_RHS_HOST || r.rhs == SEM_RHS_MANUFACTURED, "unknown rhs %d", r.rhs);
  SEM_REQUIRE(r.rhs != SEM_RHS_HOST || r.b != nullptr, "SEM_RHS_HOST needs b");
  SEM_REQUIRE(r.rhs != SEM_RHS_MANUFACTURED || r.bc == SEM_DIRICHLET,
              "the manufactured right-hand side is Dirichlet");
  SEM_REQUIRE(r.solve.solver == SEM_SOLVER_FLEXCG, "batched solves are FlexCG");
  SEM_REQUIRE(r.solve.tol >= 0.0 && r.solve.max_iter >= 0, "negative tol or max_iter");
}

void check_batch_desc(const sem_batch_desc &d) {
  SEM_REQUIRE(d.cheb_degree >= 1 && d.cheb_degree <= 16, "cheb_degree outside [1, 16]");
  SEM_REQUIRE(d.smoother_dtype >= SEM_F64 && d.smoother_dtype <= SEM_BF16, "bad smoother_dtype");
  SEM_REQUIRE(d.coarse_maxit >= 0 && d.coarse_ctas >= 0, "negative coarse_maxit or coarse_ctas");
  SEM_REQUIRE(d.arena_chunk >= 0, "negative arena_chunk");
  for (int o = 0; o <= SEM_MAX_ORDER; ++o)
    SEM_REQUIRE(d.ax_fill[o] >= 0.f && d.ax_fill[o] <= 64.f, "ax_fill[%d] outside [0, 64]", o);
}

}  // namespace
}  // namespace sem

using namespace sem;

struct sem_batch {
  sem_batch_desc d{};
  int n = 0;
  std::vector<sem_request> reqs;
  DevArena arena;                  // every device buffer of the batch
  std::vector<sem_mesh *> meshes;
  std::vector<sem_pmg *> pmgs;
  std::vector<DevBuf<double> *> bufs;  // per problem: b, x
  DevBuf<double> results;          // [n][kSlots] scalar slots after a solve
  double *pinned = nullptr;        // host copy of results
  cudaStream_t cs = nullptr;       // capture stream
  cudaGraphExec_t exec = nullptr;
  int graph_nodes = 0;
  double setup_ms = 0.0;
  ~sem_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (cs) cudaStreamDestroy(cs);
    for (sem_pmg *p : pmgs)
      if (p) sem_pmg_destroy(p);
    for (sem_mesh *m : meshes)
      if (m) sem_mesh_destroy(m);
    for (DevBuf<double> *b : bufs) delete b;
    if (pinned) cudaFreeHost(pinned);
    results.release();
    // the arena (a member) frees its chunks last
  }
  double *b(int i) { return bufs[2 * i]->p; }
  double *x(int i) { return bufs[2 * i + 1]->p; }

  sem_pmg_desc pmg_desc(int i) const {
    const std::vector<int32_t> ord = batch_orders(reqs[i].N);
    sem_pmg_desc pd{};
    pd.nlevels = (int32_t)ord.size();
    for (size_t l = 0; l < ord.size(); ++l) pd.orders[l] = ord[l];
    pd.cheb_degree = d.cheb_degree;
    pd.lanczos_steps = 20;
    pd.seed = 0;
    pd.smoother_dtype = d.smoother_dtype;
    pd.coarse_tol = d.coarse_tol;
    pd.coarse_maxit = d.coarse_maxit;
    pd.coarse_mode = SEM_COARSE_MG;
    pd.smoother = SEM_SMOOTH_JACOBI;
    pd.coarse_ctas = d.coarse_ctas > 0 ? d.coarse_ctas : 1;
    return pd;
  }

  // The FP32 operator's work split of every level of problem i.
  void apply_fill(int i) {
    std::vector<Level *> levels{&meshes[i]->fine};
    for (auto &q : pmgs[i]->levp)
      if (q && q->L && q->L != &meshes[i]->fine) levels.push_back(q->L);
    for (Level *L : levels) {
      const float f = d.ax_fill[L->t.N];
      L->ax32_fill = f > 0.f ? f : 2.0f;
    }
  }

  // One graph over the problems in `which`: every problem's solve as an
  // independent branch, each followed by the copy of its scalar slots.
  void capture(const std::vector<int> &which) {
    if (exec) {
      SEM_CHECK_CUDA(cudaGraphExecDestroy(exec));
      exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    SEM_CHECK_CUDA(cudaGraphCreate(&g, 0));
    struct GraphGuard {
      cudaGraph_t g;
      ~GraphGuard() { if (g) cudaGraphDestroy(g); }
    } gg{g};
    // largest problems first: the graph's independent branches start in about
    // the order they were added, and the batch ends with its slowest solve
    std::vector<int> order(which);
    auto work = [&](int i) {
      const sem_request &r = reqs[i];
      return (double)r.ex * r.ey * r.ez * std::pow((double)(r.N + 1), 3);
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
    for (int i : order) {
      apply_fill(i);
      const sem_solve_desc &s = reqs[i].solve;
      cudaGraphNode_t end =
          capture_flexcg(meshes[i], pmgs[i], b(i), x(i), s.tol, s.max_iter, g, cs);
      capture_slots_copy(meshes[i], results.p + (size_t)i * kSlots, g, end, cs);
    }
    size_t nodes = 0;
    SEM_CHECK_CUDA(cudaGraphGetNodes(g, nullptr, &nodes));
    graph_nodes = (int)nodes;
    SEM_CHECK_CUDA(cudaGraphInstantiate(&exec, g, 0));
  }

  // Launch the graph, read every captured problem's state; fills infos of
  // the problems in `which` (indexed like reqs).  Returns the first failing
  // status (SEM_OK if all converged).
  sem_status launch(const std::vector<int> &which, sem_solve_info *infos, cudaStream_t st,
                    bool copy_x) {
    SEM_CHECK_CUDA(cudaGraphLaunch(exec, st));
    SEM_CHECK_CUDA(cudaMemcpyAsync(pinned, results.p, (size_t)n * kSlots * sizeof(double),
                                   cudaMemcpyDeviceToHost, st));
    if (copy_x)
      for (int i : which)
        if (reqs[i].x)
          SEM_CHECK_CUDA(cudaMemcpyAsync(reqs[i].x, x(i),
                                         meshes[i]->fine.t.nl * sizeof(double),
                                         cudaMemcpyDeviceToHost, st));
    SEM_CHECK_CUDA(cudaStreamSynchronize(st));
    sem_status first = SEM_OK;
    for (int i : which) {
      sem_solve_info info{};
      sem_status s = flexcg_graph_result(pinned + (size_t)i * kSlots, info);
      if (mesh_take_wait_errors(meshes[i], pmgs[i], st)) {
        s = SEM_ETIMEOUT;
        info.status = SEM_ETIMEOUT;
      }
      if (infos) infos[i] = info;
      if (s != SEM_OK && first == SEM_OK) first = s;
    }
    return first;
  }
};

namespace {

template <typename F>
sem_status batch_guard(F &&f) {
  try {
    f();
    return SEM_OK;
  } catch (const Failure &e) {
    return e.status;
  } catch (const std::bad_alloc &) {
    set_error_message("host allocation failed");
    return SEM_ENOMEM;
  } catch (...) {
    set_error_message("unexpected internal error");
    return SEM_ECUDA;
  }
}

std::vector<int> all_of(int n) {
  std::vector<int> v(n);
  for (int i = 0; i < n; ++i) v[i] = i;
  return v;
}

}  // namespace

extern "C" {

sem_status sem_batch_create(const sem_batch_desc *desc, const sem_request *reqs, int32_t n,
                            void *stream, sem_batch **out) {
  return batch_guard([&] {
    SEM_REQUIRE(desc && reqs && out, "null argument");
    *out = nullptr;
    SEM_REQUIRE(n >= 1 && n <= 4096, "batch size %d outside [1, 4096]", n);
    check_batch_desc(*desc);
    for (int32_t i = 0; i < n; ++i) check_batch_request(reqs[i]);
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = (cudaStream_t)stream;
    std::unique_ptr<sem_batch> B(new sem_batch());
    B->d = *desc;
    B->n = n;
    B->reqs.assign(reqs, reqs + n);
    for (auto &r : B->reqs) r.b = nullptr;  // host right-hand sides are copied below
    if (desc->arena_chunk > 0) B->arena.chunk = (size_t)desc->arena_chunk;
    SEM_CHECK_CUDA(cudaStreamCreateWithFlags(&B->cs, cudaStreamNonBlocking));
    SEM_CHECK_CUDA(cudaMallocHost(&B->pinned, (size_t)n * kSlots * sizeof(double)));
    {
      ArenaScope scope(&B->arena);
      B->results.alloc((size_t)n * kSlots);
      B->meshes.assign(n, nullptr);
      B->pmgs.assign(n, nullptr);
      for (int32_t i = 0; i < n; ++i) {
        const sem_request &r = reqs[i];
        sem_mesh_desc md{};
        md.ex = r.ex;
        md.ey = r.ey;
        md.ez = r.ez;
        md.N = r.N;
        md.jitter = r.jitter;
        md.seed = r.seed;
        md.bc = r.bc;
        md.geom = SEM_GEOM_STORED;
        md.verts = nullptr;
        md.f64_arith = SEM_ARITH_PAIR;
        sem_status s = sem_mesh_create(&md, st, &B->meshes[i]);
        if (s != SEM_OK) fail(s, "batch problem %d: %s", i, sem_last_error());
        const sem_pmg_desc pd = B->pmg_desc(i);
        s = sem_pmg_setup(B->meshes[i], &pd, st, &B->pmgs[i]);
        if (s != SEM_OK) fail(s, "batch problem %d: %s", i, sem_last_error());
        const Level &L = B->meshes[i]->fine;
        const int64_t nl = L.t.nl;
        DevBuf<double> *bb = new DevBuf<double>();
        B->bufs.push_back(bb);
        DevBuf<double> *xx = new DevBuf<double>();
        B->bufs.push_back(xx);
        bb->alloc(nl);
        xx->alloc(nl);
        if (r.rhs == SEM_RHS_MANUFACTURED) {
          DevBuf<double> tmp;
          tmp.alloc(4 * (size_t)nl);
          build_manufactured_rhs(L, bb->p, tmp.p, st);
        } else {
          SEM_CHECK_CUDA(cudaMemcpyAsync(bb->p, r.b, nl * sizeof(double), cudaMemcpyHostToDevice,
                                         st));
          mesh_check_rhs(B->meshes[i], bb->p, st);  // mean-free under Neumann
        }
      }
      SEM_CHECK_CUDA(cudaStreamSynchronize(st));
      // One standalone solve per distinct order runs every kernel the graph
      // will hold once (function attributes and occupancy queries happen
      // outside the capture).
      std::set<int> seen;
      for (int32_t i = 0; i < n; ++i) {
        if (!seen.insert(reqs[i].N).second) continue;
        B->apply_fill(i);
        sem_solve_desc sd = reqs[i].solve;
        sd.zero_guess = 1;
        sd.use_graph = 0;
        sd.check_every = 1;
        sem_solve_info info{};
        const sem_status s = sem_solve(B->meshes[i], B->pmgs[i], B->b(i), B->x(i), &sd, &info, st);
        if (s != SEM_OK && s != SEM_ENOTCONV)
          fail(s, "batch problem %d (warm-up solve): %s", i, sem_last_error());
      }
      B->capture(all_of(n));
    }
    SEM_CHECK_CUDA(cudaStreamSynchronize(st));
    B->setup_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = B.release();
  });
}

sem_status sem_batch_solve(sem_batch *batch, sem_solve_info *infos, void *stream) {
  sem_status result = SEM_OK;
  const sem_status st = batch_guard([&] {
    SEM_REQUIRE(batch != nullptr, "null batch");
    SEM_REQUIRE(batch->exec != nullptr, "batch has no graph");
    result = batch->launch(all_of(batch->n), infos, (cudaStream_t)stream, true);
    if (result == SEM_ENOTCONV) set_error_message("a batched solve reached max_iter");
    else if (result == SEM_ENUMERIC) set_error_message("NaN or Inf in a batched solve");
    else if (result == SEM_ETIMEOUT)
      set_error_message("a bounded wait in a kernel ran out during the batch");
  });
  return st != SEM_OK ? st : result;
}

sem_status sem_batch_info(const sem_batch *batch, size_t *dev_bytes, int32_t *graph_nodes,
                          double *setup_ms) {
  return batch_guard([&] {
    SEM_REQUIRE(batch != nullptr, "null batch");
    if (dev_bytes) *dev_bytes = batch->arena.reserved;
    if (graph_nodes) *graph_nodes = batch->graph_nodes;
    if (setup_ms) *setup_ms = batch->setup_ms;
  });
}

sem_status sem_batch_pmg_desc(const sem_batch *batch, int32_t i, sem_pmg_desc *out) {
  return batch_guard([&] {
    SEM_REQUIRE(batch != nullptr && out != nullptr, "null argument");
    SEM_REQUIRE(i >= 0 && i < batch->n, "problem %d outside [0, %d)", i, batch->n);
    *out = batch->pmg_desc(i);
  });
}

sem_status sem_batch_x(const sem_batch *batch, int32_t i, const double **x_dev) {
  return batch_guard([&] {
    SEM_REQUIRE(batch != nullptr && x_dev != nullptr, "null argument");
    SEM_REQUIRE(i >= 0 && i < batch->n, "problem %d outside [0, %d)", i, batch->n);
    *x_dev = const_cast<sem_batch *>(batch)->x(i);
  });
}

sem_status sem_batch_destroy(sem_batch *batch) {
  return batch_guard([&] { delete batch; });
}

sem_status sem_batch_autotune(sem_batch *batch, const float *candidates, int32_t ncand,
                              int32_t reps, void *stream, float *chosen, double *best_ms) {
  return batch_guard([&] {
    SEM_REQUIRE(batch && candidates && chosen && best_ms, "null argument");
    SEM_REQUIRE(ncand >= 1 && ncand <= 32 && reps >= 1 && reps <= 100, "bad ncand or reps");
    for (int32_t c = 0; c < ncand; ++c)
      SEM_REQUIRE(candidates[c] > 0.f && candidates[c] <= 64.f, "candidate %d outside (0, 64]", c);
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    SEM_CHECK_CUDA(cudaEventCreate(&e0));
    SEM_CHECK_CUDA(cudaEventCreate(&e1));
    struct EvGuard {
      cudaEvent_t a, b;
      ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } guard{e0, e1};
    const std::vector<int> everyone = all_of(batch->n);
    // median time of one launch of the whole batch with the current split
    auto time_batch = [&]() {
      batch->capture(everyone);
      batch->launch(everyone, nullptr, st, false);  // warm-up
      std::vector<float> t(reps);
      for (int32_t k = 0; k < reps; ++k) {
        SEM_CHECK_CUDA(cudaEventRecord(e0, st));
        SEM_CHECK_CUDA(cudaGraphLaunch(batch->exec, st));
        SEM_CHECK_CUDA(cudaEventRecord(e1, st));
        SEM_CHECK_CUDA(cudaEventSynchronize(e1));
        SEM_CHECK_CUDA(cudaEventElapsedTime(&t[k], e0, e1));
      }
      std::sort(t.begin(), t.end());
      return (double)t[reps / 2];
    };
    // problems grouped by fine order: the levels of a class (orders N, N/2)
    // share one value.  Coordinate descent on the whole batch, the problems
    // of every class running beside the others as in use: one class at a
    // time tries every candidate and keeps the fastest whole-batch time.
    // A candidate replaces the current value only when it is faster by more
    // than the margin (launch-to-launch variation of a batch is a few per
    // cent), and the tuned split must beat the starting one again, timed
    // alternately with it, or the starting split is kept.
    constexpr double kMargin = 0.02;
    std::set<int> classes;
    for (int i = 0; i < batch->n; ++i) classes.insert(batch->reqs[i].N);
    float start[SEM_MAX_ORDER + 1];
    std::copy(batch->d.ax_fill, batch->d.ax_fill + SEM_MAX_ORDER + 1, start);
    double best = time_batch();
    for (int N : classes) {
      const std::vector<int32_t> ord = batch_orders(N);
      const float keep = batch->d.ax_fill[N];
      float best_f = keep;
      for (int32_t c = 0; c < ncand; ++c) {
        if (candidates[c] == keep) continue;
        for (int o : ord) batch->d.ax_fill[o] = candidates[c];
        const double t = time_batch();
        if (t < best * (1.0 - kMargin)) {
          best = t;
          best_f = candidates[c];
        }
      }
      for (int o : ord) batch->d.ax_fill[o] = best_f;
    }
    if (!std::equal(start, start + SEM_MAX_ORDER + 1, batch->d.ax_fill)) {
      float tuned[SEM_MAX_ORDER + 1];
      std::copy(batch->d.ax_fill, batch->d.ax_fill + SEM_MAX_ORDER + 1, tuned);
      double t_tuned = 0.0, t_start = 0.0;
      for (int r = 0; r < 2; ++r) {
        std::copy(tuned, tuned + SEM_MAX_ORDER + 1, batch->d.ax_fill);
        t_tuned += time_batch();
        std::copy(start, start + SEM_MAX_ORDER + 1, batch->d.ax_fill);
        t_start += time_batch();
      }
      const float *keep_fill = t_tuned < t_start * (1.0 - kMargin) ? tuned : start;
      std::copy(keep_fill, keep_fill + SEM_MAX_ORDER + 1, batch->d.ax_fill);
    }
    for (int o = 0; o <= SEM_MAX_ORDER; ++o) chosen[o] = batch->d.ax_fill[o];
    *best_ms = time_batch();
  });
}

}  // extern "C"
