// capi.cu -- the C ABI of include/sem.h: argument checks, error reporting,
// mesh and pMG handles, and the host loops of the Krylov solvers.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>

#include "common.cuh"
#include "kernels.cuh"
#include "pmg.cuh"
#include "trace.cuh"

namespace sem {

static thread_local std::string g_error;

void set_error_message(const char *msg) { g_error = msg ? msg : ""; }

[[noreturn]] void fail(sem_status st, const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_error = buf;
  throw Failure{st};
}

template <typename F>
static sem_status guarded(F &&f) {
  try {
    f();
    return SEM_OK;
  } catch (const Failure &e) {
    return e.status;
  } catch (const std::bad_alloc &) {
    g_error = "host allocation failed";
    return SEM_ENOMEM;
  } catch (...) {
    g_error = "unexpected internal error";
    return SEM_ECUDA;
  }
}

// Unit-cube lattice with interior vertices moved by splitmix64 offsets
// (see sem_mesh_desc).
static std::vector<double> builtin_vertices(int ex, int ey, int ez, double jitter, uint64_t seed) {
  const size_t nv = (size_t)(ex + 1) * (ey + 1) * (ez + 1);
  std::vector<double> v(3 * nv);
  const int cnt[3] = {ex, ey, ez};
  for (int c = 0; c <= ez; ++c)
    for (int b = 0; b <= ey; ++b)
      for (int a = 0; a <= ex; ++a) {
        const size_t id = a + (size_t)(ex + 1) * (b + (size_t)(ey + 1) * c);
        const int idx[3] = {a, b, c};
        const bool interior = a > 0 && a < ex && b > 0 && b < ey && c > 0 && c < ez;
        for (int m = 0; m < 3; ++m) {
          double x = (double)idx[m] / (double)cnt[m];
          if (interior) {
            uint64_t z = seed + (uint64_t)(3 * id + m + 1) * 0x9E3779B97F4A7C15ull;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
            double off = ((2.0 * u - 1.0) * jitter) / (double)cnt[m];
            x = x + off;
          }
          v[3 * id + m] = x;
        }
      }
  return v;
}

// Work vectors of the outer solver, each starting on a 256-byte boundary.
static size_t work_stride(const sem_mesh *M) { return ((size_t)M->fine.t.nl + 31) / 32 * 32; }

static void ensure_work(sem_mesh *M) {
  if (M->work.p) return;
  M->work.alloc(4 * work_stride(M));
}

static double *slot(sem_mesh *M, int s) { return M->scal.p + s; }

static void read_scalars(sem_mesh *M, int count, cudaStream_t st) {
  SEM_CHECK_CUDA(cudaMemcpyAsync(M->pinned, M->scal.p, count * sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
  SEM_CHECK_CUDA(cudaStreamSynchronize(st));
}

// Under Neumann the right-hand side must be mean-free (Sec. 3: the pressure
// Poisson problem with Neumann conditions is consistent only then).
static void check_neumann_rhs(sem_mesh *M, const double *b, cudaStream_t st) {
  const Topo &t = M->fine.t;
  if (t.bc != SEM_NEUMANN) return;
  launch_sum(t, M->red, b, slot(M, 6), st);
  launch_dot(t, M->red, b, b, slot(M, 0), st);
  read_scalars(M, 8, st);
  double s = M->pinned[6], bb = M->pinned[0];
  SEM_REQUIRE(std::fabs(s) <= 1e-10 * std::sqrt((double)t.ng) * std::sqrt(bb) || bb == 0.0,
              "Neumann right-hand side is not mean-free (sum %.3e, norm %.3e)", s,
              std::sqrt(bb));
}

// A kernel whose bounded wait ran out (a bulk copy that never completed)
// sets its level's flag and leaves the rest of its work undone.  After a
// solve's last synchronisation the flags of every level it used are read and
// cleared; a set flag makes the solve's status SEM_ETIMEOUT.
static bool take_wait_errors(sem_mesh *M, sem_pmg *P, cudaStream_t st) {
  std::vector<sem::Level *> levels{&M->fine};
  if (P)
    for (auto &q : P->levp)
      if (q && q->L && q->L != &M->fine) levels.push_back(q->L);
  bool any = false;
  for (sem::Level *L : levels) {
    if (!L->err.p) continue;
    int v = 0;
    SEM_CHECK_CUDA(cudaMemcpyAsync(&v, L->err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    SEM_CHECK_CUDA(cudaStreamSynchronize(st));
    if (v != 0) {
      any = true;
      SEM_CHECK_CUDA(cudaMemsetAsync(L->err.p, 0, sizeof(int), st));
    }
  }
  if (any) SEM_CHECK_CUDA(cudaStreamSynchronize(st));
  return any;
}

static sem_status report_wait_errors(sem_mesh *M, sem_pmg *P, cudaStream_t st,
                                     sem_solve_info &info, sem_status status) {
  if (!take_wait_errors(M, P, st)) return status;
  info.status = SEM_ETIMEOUT;
  set_error_message("a bounded wait in a kernel ran out (a bulk copy did not complete); "
                    "the solve's results are incomplete");
  return SEM_ETIMEOUT;
}

// Flexible GMRES(m) (Sec. 3: the GMRES alternative to FlexCG; Sec. 5: few
// vectors, classical Gram-Schmidt with one reduction for all coefficients of
// a step).  Right preconditioning by one pMG V-cycle (or Jacobi without pmg);
// the preconditioned vectors z_j are kept because the V-cycle may vary, and
// x = x0 + Z y (Saad, Alg. 9.6).  The small least-squares problem lives on
// the host (Givens rotations, as in the oracle); per step the device runs the
// preconditioner, the FP64 operator, one multi-dot <w, v_i>, one fused
// subtract-and-norm pass and a scaling, and the host reads one Hessenberg
// column.  A cycle ends when the least-squares residual meets the tolerance
// or after m steps; x is then updated and its residual recomputed, which
// decides convergence (restarting from it otherwise).
static sem_status run_fgmres(sem_mesh *M, sem_pmg *P, const double *b, double *x,
                             const sem_solve_desc &d, sem_solve_info &info, cudaStream_t st,
                             bool x_zero = false, bool check_rhs = true) {
  const Level &L = M->fine;
  const Topo &t = L.t;
  const int m = d.restart > 0 ? d.restart : 20;
  SEM_REQUIRE(m >= 1 && m <= kMaxKrylov, "restart %d outside [1, %d]", m, kMaxKrylov);
  const size_t ws = work_stride(M);
  if (M->krylov_m < m) {
    M->krylov.alloc((size_t)(2 * m + 2) * ws);
    M->krylov_m = m;
  }
  if (!M->kred.partials.p) M->kred.init(kVecMaxBlocks, kMaxKrylov + 1);
  if (!M->kscal.p) M->kscal.alloc(kMaxKrylov + 4);
  if (!M->kpinned) SEM_CHECK_CUDA(cudaMallocHost(&M->kpinned, (kMaxKrylov + 4) * sizeof(double)));
  const int cap = M->krylov_m;
  double *V = M->krylov.p, *Z = V + (size_t)(cap + 1) * ws, *w = Z + (size_t)cap * ws;
  double *h = M->kscal.p, *nrm2 = h + kMaxKrylov + 1;
  cudaEvent_t e0, e1;
  SEM_CHECK_CUDA(cudaEventCreate(&e0));
  SEM_CHECK_CUDA(cudaEventCreate(&e1));
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); }
  } guard{e0, e1};
  SEM_CHECK_CUDA(cudaEventRecord(e0, st));
  if (d.zero_guess && !x_zero) {
    SEM_CHECK_CUDA(cudaMemsetAsync(x, 0, t.nl * sizeof(double), st));
    x_zero = true;
  }
  if (check_rhs) check_neumann_rhs(M, b, st);
  // r0 = b - A x into V_0 (r0 = b when x is known to be zero), with <b, b>, <r0, r0>
  if (!x_zero) apply_assembled<double>(L, x, w, st);
  launch_cg_start(t, M->red, b, x_zero ? nullptr : w, nullptr, V, nullptr, nullptr, slot(M, 0),
                  slot(M, 1), slot(M, 2), st);
  read_scalars(M, 8, st);
  const double bb = M->pinned[0];
  double beta = std::sqrt(M->pinned[1]);
  info.bnorm = std::sqrt(bb);
  info.res0 = beta;
  const double target = d.tol * info.bnorm;
  sem_status status = SEM_ENOTCONV;
  if (!(beta == beta) || !(bb == bb)) status = SEM_ENUMERIC;
  else if (beta <= target) status = SEM_OK;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  int k = 0;
  while (status == SEM_ENOTCONV && k < d.max_iter) {
    launch_scale(t.nl, 1.0 / beta, V, st);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int cols = 0;
    for (int j = 0; j < m && k < d.max_iter; ++j) {
      double *vj = V + (size_t)j * ws, *zj = Z + (size_t)j * ws, *vn = V + (size_t)(j + 1) * ws;
      if (P) pmg_vcycle(P, vj, zj, st);
      else launch_mul(t.nl, L.dinv64.p, vj, zj, st);
      apply_assembled<double>(L, zj, w, st);
      // classical Gram-Schmidt: every coefficient from the same w
      launch_multi_dot(t, M->kred, w, V, ws, j + 1, h, st);
      launch_orth_update(t, M->kred, w, V, ws, j + 1, h, vn, nrm2, st);
      SEM_CHECK_CUDA(cudaMemcpyAsync(M->kpinned, h, (kMaxKrylov + 2) * sizeof(double),
                                     cudaMemcpyDeviceToHost, st));
      SEM_CHECK_CUDA(cudaStreamSynchronize(st));
      const double hn = std::sqrt(std::max(M->kpinned[kMaxKrylov + 1], 0.0));
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = M->kpinned[i];
      H[(size_t)(j + 1) * m + j] = hn;
      if (!std::isfinite(hn) || !std::isfinite(M->kpinned[j])) {
        status = SEM_ENUMERIC;
        break;
      }
      for (int i = 0; i < j; ++i) {
        const double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      const double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
      const double dd = std::sqrt(a * a + c * c);
      cs[j] = dd > 0.0 ? a / dd : 1.0;
      sn[j] = dd > 0.0 ? c / dd : 0.0;
      H[(size_t)j * m + j] = dd;
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++k;
      cols = j + 1;
      if (std::fabs(g[j + 1]) <= target || hn == 0.0) break;
      if (j + 1 < m && k < d.max_iter) launch_scale(t.nl, 1.0 / hn, vn, st);
    }
    if (status == SEM_ENUMERIC) break;
    // y = R^-1 g by back substitution; x += Z y
    for (int i = cols - 1; i >= 0; --i) {
      double s = g[i];
      for (int q = i + 1; q < cols; ++q) s -= H[(size_t)i * m + q] * y[q];
      y[i] = s / H[(size_t)i * m + i];
    }
    launch_combine(t.nl, Z, ws, cols, y.data(), x, st);
    apply_assembled<double>(L, x, w, st);
    launch_cg_start(t, M->red, b, w, nullptr, V, nullptr, nullptr, slot(M, 0), slot(M, 1),
                    slot(M, 2), st);
    read_scalars(M, 8, st);
    beta = std::sqrt(M->pinned[1]);
    if (!(beta == beta) || std::isinf(beta)) status = SEM_ENUMERIC;
    else if (beta <= target) status = SEM_OK;
  }
  SEM_CHECK_CUDA(cudaEventRecord(e1, st));
  SEM_CHECK_CUDA(cudaEventSynchronize(e1));
  info.iters = k;
  info.res = beta;
  float ms = 0.f;
  SEM_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  info.time_ms = ms;
  info.status = status;
  if (status == SEM_ENOTCONV)
    set_error_message("solver reached max_iter before the tolerance");
  else if (status == SEM_ENUMERIC)
    set_error_message("NaN or Inf in the solver residual");
  return report_wait_errors(M, P, st, info, status);
}

// Flexible CG steps (Sec. 3).  The V-cycle reads its input from, and leaves
// its output in, the fine level's own buffers (FP32 for an FP32 smoother):
// cg_update writes the V-cycle input beside r, and the direction update, the
// dots and the operator read the FP32 output directly (widened exactly), so
// no separate conversion passes run.  With the stored-factor pair operator
// <p, Ap> is reduced inside the operator kernel.
// Scalar slots: 0 bb, 1 rr, 2 rho = <z,r>, 4 <p,Ap>, 5 <z,w>, 7 unused.
static bool flex_fused(const Level &L) {
  return L.geom == SEM_GEOM_STORED && L.arith == SEM_ARITH_PAIR;
}

// p = z (first) or p = z - (<z,w>/<p,w>) p;  w = mask gs(A p);  slot 4 = <p, w>
static void flex_operator(sem_mesh *M, const VcycleIO &io, double *p, double *w, bool first,
                          cudaStream_t st) {
  const Level &L = M->fine;
  const Topo &t = L.t;
  if (first) {
    if (io.out32) launch_convert<float, double>(t.nl, io.out32, p, st);
    else launch_convert<double, double>(t.nl, io.out64, p, st);
  } else if (io.out32) {
    launch_cg_direction(t.nl, slot(M, 5), slot(M, 4), -1.0, io.out32, p, nullptr, st);
  } else {
    launch_cg_direction(t.nl, slot(M, 5), slot(M, 4), -1.0, io.out64, p, nullptr, st);
  }
  if (flex_fused(L)) {
    launch_ax_pair_dot(L, p, w, slot(M, 4), M->red, st);
    launch_planes_assemble<double>(L, w, st);
  } else {
    apply_assembled<double>(L, p, w, st);
    launch_dot(t, M->red, p, w, slot(M, 4), st);
  }
}

// x += alpha p, r -= alpha w, rr (slot 1), and the V-cycle input = r
static void flex_update(sem_mesh *M, const VcycleIO &io, const double *p, const double *w,
                        double *x, double *r, cudaStream_t st) {
  launch_cg_update(M->fine.t, M->red, slot(M, 2), slot(M, 4), p, w, nullptr, x, r, nullptr,
                   slot(M, 1), slot(M, 7), nullptr, st, io.in32, io.in64);
}

// z = V-cycle(r) (in the level's buffers); slot 2 = <z,r>, slot 5 = <z,w>
static void flex_precondition(sem_mesh *M, sem_pmg *P, const VcycleIO &io, const double *r,
                              const double *w, cudaStream_t st) {
  pmg_vcycle_core(P, st);
  if (io.out32) launch_flex_dots(M->fine.t, M->red, io.out32, r, w, slot(M, 2), slot(M, 5), st);
  else launch_flex_dots(M->fine.t, M->red, io.out64, r, w, slot(M, 2), slot(M, 5), st);
}

// The FlexCG loop as a CUDA graph: one while node whose body is one pass of
// the iteration, beginning with the preconditioner of the previous
// iteration (V-cycle and the two dots) and ending with this iteration's
// direction, operator, step and stopping test (launch_graph_stop, which sets
// the loop condition): the same kernels as the host-driven loop, in the same
// order.  The body bakes in the
// mesh's work vectors, the pMG's buffers and x; the mesh keeps one
// executable graph and captures again when the pMG or x changes.
static void ensure_graph(sem_mesh *M, sem_pmg *P, double *x) {
  if (M->graph && M->graph_pmg == P->serial && M->graph_x == x) return;
  if (M->graph) {
    SEM_CHECK_CUDA(cudaGraphExecDestroy(M->graph));
    M->graph = nullptr;
  }
  if (!M->cstream) SEM_CHECK_CUDA(cudaStreamCreateWithFlags(&M->cstream, cudaStreamNonBlocking));
  const size_t ws = work_stride(M);
  double *r = M->work.p, *z = r + ws, *p = z + ws, *w = p + ws;
  cudaStream_t cs = M->cstream;
  cudaGraph_t g = nullptr;
  SEM_CHECK_CUDA(cudaGraphCreate(&g, 0));
  struct GraphGuard {
    cudaGraph_t g;
    ~GraphGuard() { if (g) cudaGraphDestroy(g); }
  } gg{g};
  cudaGraphConditionalHandle h;
  SEM_CHECK_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  SEM_CHECK_CUDA(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  SEM_CHECK_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal));
  std::map<std::string, int64_t> tally;  // kernels of one pass per trace class
  trace_tally_begin(&tally);
  try {
    const VcycleIO io = pmg_io(P);
    flex_precondition(M, P, io, r, w, cs);
    flex_operator(M, io, p, w, false, cs);
    flex_update(M, io, p, w, x, r, cs);
    launch_graph_stop(slot(M, 1), slot(M, 8), h, cs);
  } catch (...) {
    trace_tally_end();
    cudaGraph_t tmp = nullptr;
    cudaStreamEndCapture(cs, &tmp);
    cudaGetLastError();
    throw;
  }
  trace_tally_end();
  cudaGraph_t out = nullptr;
  SEM_CHECK_CUDA(cudaStreamEndCapture(cs, &out));
  size_t nodes = 0;
  SEM_CHECK_CUDA(cudaGraphGetNodes(body, nullptr, &nodes));
  std::vector<cudaGraphNode_t> list(nodes);
  if (nodes) SEM_CHECK_CUDA(cudaGraphGetNodes(body, list.data(), &nodes));
  int kernels = 0;
  for (cudaGraphNode_t n : list) {
    cudaGraphNodeType ty;
    SEM_CHECK_CUDA(cudaGraphNodeGetType(n, &ty));
    kernels += ty == cudaGraphNodeTypeKernel;
  }
  SEM_CHECK_CUDA(cudaGraphInstantiate(&M->graph, g, 0));
  M->graph_pmg = P->serial;
  M->graph_x = x;
  M->graph_kernels = kernels;
  M->graph_tally = std::move(tally);
}

// Nodes of `g` that no other node of `g` depends on (the end of what a
// capture appended, when the capture was one sequence).
static std::vector<cudaGraphNode_t> graph_sinks(cudaGraph_t g) {
  size_t n = 0;
  SEM_CHECK_CUDA(cudaGraphGetNodes(g, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n), sinks;
  if (n) SEM_CHECK_CUDA(cudaGraphGetNodes(g, nodes.data(), &n));
  for (cudaGraphNode_t v : nodes) {
    size_t m = 0;
    SEM_CHECK_CUDA(cudaGraphNodeGetDependentNodes(v, nullptr, nullptr, &m));
    if (m == 0) sinks.push_back(v);
  }
  return sinks;
}

// Capture into `g` one sequence run on stream cs, after the nodes `deps` of
// `g`; returns the nodes it added that nothing depends on.
template <typename F>
static std::vector<cudaGraphNode_t> capture_into(cudaGraph_t g, cudaStream_t cs,
                                                 const std::vector<cudaGraphNode_t> &deps,
                                                 F &&work) {
  size_t n0 = 0;
  SEM_CHECK_CUDA(cudaGraphGetNodes(g, nullptr, &n0));
  std::vector<cudaGraphNode_t> old(n0);
  if (n0) SEM_CHECK_CUDA(cudaGraphGetNodes(g, old.data(), &n0));
  SEM_CHECK_CUDA(cudaStreamBeginCaptureToGraph(cs, g, deps.empty() ? nullptr : deps.data(),
                                               nullptr, deps.size(),
                                               cudaStreamCaptureModeThreadLocal));
  try {
    work();
  } catch (...) {
    cudaGraph_t tmp = nullptr;
    cudaStreamEndCapture(cs, &tmp);
    cudaGetLastError();
    throw;
  }
  cudaGraph_t out = nullptr;
  SEM_CHECK_CUDA(cudaStreamEndCapture(cs, &out));
  std::vector<cudaGraphNode_t> sinks;
  for (cudaGraphNode_t v : graph_sinks(g))
    if (std::find(old.begin(), old.end(), v) == old.end()) sinks.push_back(v);
  return sinks;
}

// A conditional node of type ty in g after deps; returns its body graph and,
// in *node, the node.
static cudaGraph_t add_conditional(cudaGraph_t g, const std::vector<cudaGraphNode_t> &deps,
                                   cudaGraphConditionalHandle h, cudaGraphConditionalNodeType ty,
                                   cudaGraphNode_t *node) {
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = ty;
  np.conditional.size = 1;
  SEM_CHECK_CUDA(cudaGraphAddNode(node, g, deps.empty() ? nullptr : deps.data(), nullptr,
                                  deps.size(), &np));
  return np.conditional.phGraph_out[0];
}

// A whole FlexCG solve from x = 0 (Sec. 3), run by the device, appended to
// graph `g` as a branch of its own (no dependencies on the graph's other
// nodes): the kernels of run_solve with use_graph and zero_guess, in the same
// order, the host's stopping tests replaced by device ones (the arm kernel
// after the start, the stop kernel after every iteration).  The branch is
//   memset x, start (r = b, <b,b>, <r,r>), arm -> IF(iterations due) {
//     V-cycle of r, <z,r>, iteration 1, stop -> WHILE(not done) {
//       V-cycle, dots, direction, operator, update, stop } }
// so its results equal those of sem_solve bit for bit.  The state is left in
// the mesh's scalar slots: 0 <b,b>, 1 <r,r>, 8 tol^2 <b,b>, 9 max_iter,
// 10 iterations, 11 stopping state (1 done, 2 NaN/Inf), 12 initial <r,r>
// (flexcg_graph_result reads them).  Returns the branch's last node.  The
// work vectors are allocated before the capture begins.
cudaGraphNode_t capture_flexcg(sem_mesh *M, sem_pmg *P, const double *b, double *x, double tol,
                               int maxit, cudaGraph_t g, cudaStream_t cs) {
  const Level &L = M->fine;
  const Topo &t = L.t;
  ensure_work(M);
  const size_t ws = work_stride(M);
  double *r = M->work.p, *z = r + ws, *p = z + ws, *w = p + ws;
  cudaGraphConditionalHandle hif, hwhile;
  SEM_CHECK_CUDA(cudaGraphConditionalHandleCreate(&hif, g, 0, cudaGraphCondAssignDefault));
  std::vector<cudaGraphNode_t> head = capture_into(g, cs, {}, [&] {
    SEM_CHECK_CUDA(cudaMemsetAsync(x, 0, t.nl * sizeof(double), cs));
    launch_cg_start(t, M->red, b, nullptr, nullptr, r, z, p, slot(M, 0), slot(M, 1), slot(M, 2),
                    cs);
    launch_graph_arm_full(slot(M, 0), slot(M, 1), slot(M, 8), tol, maxit, hif, cs);
  });
  cudaGraphNode_t if_node, while_node;
  cudaGraph_t body_if = add_conditional(g, head, hif, cudaGraphCondTypeIf, &if_node);
  SEM_CHECK_CUDA(
      cudaGraphConditionalHandleCreate(&hwhile, body_if, 0, cudaGraphCondAssignDefault));
  const VcycleIO io = pmg_io(P);
  std::vector<cudaGraphNode_t> first = capture_into(body_if, cs, {}, [&] {
    if (io.in32) launch_convert<double, float>(t.nl, r, io.in32, cs);
    else launch_convert<double, double>(t.nl, r, io.in64, cs);
    pmg_vcycle_core(P, cs);
    if (io.out32) launch_dot(t, M->red, io.out32, r, slot(M, 2), cs);
    else launch_dot(t, M->red, io.out64, r, slot(M, 2), cs);
    flex_operator(M, io, p, w, true, cs);
    flex_update(M, io, p, w, x, r, cs);
    launch_graph_stop(slot(M, 1), slot(M, 8), hwhile, cs);
  });
  cudaGraph_t body_while =
      add_conditional(body_if, first, hwhile, cudaGraphCondTypeWhile, &while_node);
  capture_into(body_while, cs, {}, [&] {
    flex_precondition(M, P, io, r, w, cs);
    flex_operator(M, io, p, w, false, cs);
    flex_update(M, io, p, w, x, r, cs);
    launch_graph_stop(slot(M, 1), slot(M, 8), hwhile, cs);
  });
  return if_node;
}

// Append to g, after `after`, a copy of the mesh's scalar slots 0..12 into
// dst (device) and return the copy's node.
cudaGraphNode_t capture_slots_copy(sem_mesh *M, double *dst, cudaGraph_t g, cudaGraphNode_t after,
                                   cudaStream_t cs) {
  std::vector<cudaGraphNode_t> tail = capture_into(g, cs, {after}, [&] {
    SEM_CHECK_CUDA(cudaMemcpyAsync(dst, slot(M, 0), 13 * sizeof(double),
                                   cudaMemcpyDeviceToDevice, cs));
  });
  SEM_REQUIRE(tail.size() == 1, "slot copy capture");
  return tail[0];
}

// The Neumann right-hand-side check of the solves (check_neumann_rhs).
void mesh_check_rhs(sem_mesh *M, const double *b, cudaStream_t st) { check_neumann_rhs(M, b, st); }

// Read and clear the wait flags of a mesh and its pMG (take_wait_errors).
bool mesh_take_wait_errors(sem_mesh *M, sem_pmg *P, cudaStream_t st) {
  return take_wait_errors(M, P, st);
}

// The stopping state of a solve captured by capture_flexcg, from its scalar
// slots s[0..12] (read by the caller): fills info and returns the status the
// host loop of run_solve would have returned.
sem_status flexcg_graph_result(const double *s, sem_solve_info &info) {
  const double bb = s[0], rr = s[1], tol2 = s[8];
  info.bnorm = std::sqrt(bb);
  info.res0 = std::sqrt(s[12]);
  info.res = std::sqrt(rr);
  info.iters = (int32_t)s[10];
  sem_status st;
  if (s[11] == 2.0) st = SEM_ENUMERIC;
  else st = rr <= tol2 ? SEM_OK : SEM_ENOTCONV;
  info.status = st;
  return st;
}

// Jacobi-PCG (Sec. 3) or flexible CG with one pMG V-cycle per iteration
// (Sec. 3).  Scalar slots: 0 bb, 1 rr, 2/3 rho (alternating in PCG), 4 pw,
// 5 zw, 6 sum of b, 7 unused output, 8-11 state of the graph loop.
static sem_status run_solve(sem_mesh *M, sem_pmg *P, const double *b, double *x,
                            const sem_solve_desc &d, sem_solve_info &info, cudaStream_t st,
                            bool x_zero = false, bool check_rhs = true) {
  const Level &L = M->fine;
  const Topo &t = L.t;
  const bool flex = d.solver == SEM_SOLVER_FLEXCG;
  ensure_work(M);
  const size_t ws = work_stride(M);
  double *r = M->work.p, *z = r + ws, *p = z + ws, *w = p + ws;
  cudaEvent_t e0, e1;
  SEM_CHECK_CUDA(cudaEventCreate(&e0));
  SEM_CHECK_CUDA(cudaEventCreate(&e1));
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); }
  } guard{e0, e1};
  SEM_CHECK_CUDA(cudaEventRecord(e0, st));
  if (d.zero_guess && !x_zero) {
    SEM_CHECK_CUDA(cudaMemsetAsync(x, 0, t.nl * sizeof(double), st));
    x_zero = true;
  }
  if (check_rhs) check_neumann_rhs(M, b, st);
  if (!x_zero) apply_assembled<double>(L, x, w, st);
  launch_cg_start(t, M->red, b, x_zero ? nullptr : w, flex ? nullptr : L.dinv64.p, r, z, p,
                  slot(M, 0), slot(M, 1), slot(M, 2), st);
  read_scalars(M, 8, st);
  const double bb = M->pinned[0];
  double rr = M->pinned[1];
  info.bnorm = std::sqrt(bb);
  info.res0 = std::sqrt(rr);
  info.iters = 0;
  sem_status status = SEM_ENOTCONV;
  const double tol2 = d.tol * d.tol * bb;
  if (!(rr == rr) || !(bb == bb)) status = SEM_ENUMERIC;
  else if (rr <= tol2) status = SEM_OK;
  VcycleIO io;
  if (status == SEM_ENOTCONV && flex) {
    io = pmg_io(P);
    if (io.in32) launch_convert<double, float>(t.nl, r, io.in32, st);
    else launch_convert<double, double>(t.nl, r, io.in64, st);
    pmg_vcycle_core(P, st);
    if (io.out32) launch_dot(t, M->red, io.out32, r, slot(M, 2), st);
    else launch_dot(t, M->red, io.out64, r, slot(M, 2), st);
  }
  const bool graph = flex && d.use_graph != 0;
  const int every = graph || d.check_every < 1 ? 1 : d.check_every;
  for (int it = 1; status == SEM_ENOTCONV && it <= d.max_iter; ++it) {
    if (graph && it == 2) {
      // iterations 2.. on the device: one graph launch, one read
      ensure_graph(M, P, x);
      launch_graph_arm(slot(M, 8), tol2, d.max_iter, 1, st);
      {
        // timed as a whole when the filter asks; its kernels are counted
        // per class below, from the capture's tally
        TraceScope ts("flexcg_graph", t.N, st, 0);
        SEM_CHECK_CUDA(cudaGraphLaunch(M->graph, st));
      }
      read_scalars(M, 12, st);
      const int done = (int)M->pinned[10];
      for (const auto &kv : M->graph_tally) trace_count_key(kv.first, (int64_t)(done - 1) * kv.second);
      info.iters = done;
      if (M->pinned[11] == 2.0) status = SEM_ENUMERIC;
      else if (M->pinned[1] <= tol2) status = SEM_OK;
      break;
    }
    const int cur = 2 + ((it - 1) & 1), nxt = 2 + (it & 1);
    if (flex) {
      flex_operator(M, io, p, w, it == 1, st);
      flex_update(M, io, p, w, x, r, st);
    } else {
      apply_assembled<double>(L, p, w, st);
      launch_dot(t, M->red, p, w, slot(M, 4), st);
      launch_cg_update(t, M->red, slot(M, cur), slot(M, 4), p, w, L.dinv64.p, x, r, z, slot(M, 1),
                       slot(M, nxt), nullptr, st);
    }
    info.iters = it;
    if (it % every == 0 || it == d.max_iter) {
      read_scalars(M, 8, st);
      rr = M->pinned[1];
      if (!(rr == rr) || std::isinf(rr)) { status = SEM_ENUMERIC; break; }
      if (rr <= tol2) { status = SEM_OK; break; }
    }
    if (it == d.max_iter) break;
    if (graph) continue;  // the graph begins with this iteration's V-cycle
    if (flex) flex_precondition(M, P, io, r, w, st);
    else
      launch_cg_direction(t.nl, slot(M, nxt), slot(M, cur), 1.0, (const double *)z, p, nullptr,
                          st);
  }
  SEM_CHECK_CUDA(cudaEventRecord(e1, st));
  read_scalars(M, 8, st);
  rr = M->pinned[1];
  info.res = std::sqrt(rr);
  if (status == SEM_ENOTCONV && rr <= tol2) status = SEM_OK;
  float ms = 0.f;
  SEM_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  info.time_ms = ms;
  info.status = status;
  if (status == SEM_ENOTCONV)
    set_error_message("solver reached max_iter before the tolerance");
  else if (status == SEM_ENUMERIC)
    set_error_message("NaN or Inf in the solver residual");
  return report_wait_errors(M, P, st, info, status);
}

// Projected solve (Sec. 3, "Projection is key"; the oracle's
// orc_solve_projected step by step).
static sem_status run_projected(sem_mesh *M, sem_pmg *P, sem_proj *Q, const double *b, double *x,
                                const sem_solve_desc &d, sem_solve_info &info, cudaStream_t st) {
  const Level &L = M->fine;
  const Topo &t = L.t;
  const size_t ws = work_stride(M);
  const int64_t n = t.nl;
  double *Pv = Q->P.p, *APv = Q->AP.p, *c = Q->coef.p;
  if (!M->kred.partials.p) M->kred.init(kVecMaxBlocks, kMaxKrylov + 1);
  if (!M->kpinned) SEM_CHECK_CUDA(cudaMallocHost(&M->kpinned, (kMaxKrylov + 4) * sizeof(double)));
  auto read_coef = [&](int count) {
    SEM_CHECK_CUDA(cudaMemcpyAsync(M->kpinned, c, count * sizeof(double), cudaMemcpyDeviceToHost,
                                   st));
    SEM_CHECK_CUDA(cudaStreamSynchronize(st));
    return std::vector<double>(M->kpinned, M->kpinned + count);
  };
  // the original right-hand side is checked; its projected part inherits it
  check_neumann_rhs(M, b, st);
  const int k = Q->nvec;
  // best fit xbar = P P^T b into x; bp = b - AP P^T b
  SEM_CHECK_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), st));
  SEM_CHECK_CUDA(cudaMemcpyAsync(Q->bp.p, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (k > 0) {
    launch_multi_dot(t, M->kred, b, Pv, ws, k, c, st);
    std::vector<double> cf = read_coef(k), neg(k);
    for (int i = 0; i < k; ++i) neg[i] = -cf[i];
    launch_combine(n, Pv, ws, k, cf.data(), x, st);
    launch_combine(n, APv, ws, k, neg.data(), Q->bp.p, st);
  }
  launch_dot(t, M->red, b, b, slot(M, 0), st);
  launch_dot(t, M->red, Q->bp.p, Q->bp.p, slot(M, 1), st);
  read_scalars(M, 8, st);
  const double bnorm = std::sqrt(M->pinned[0]), bpn = std::sqrt(M->pinned[1]);
  sem_status status = SEM_OK;
  SEM_CHECK_CUDA(cudaMemsetAsync(Q->dx.p, 0, n * sizeof(double), st));
  info.iters = 0;
  info.res = bpn;
  info.time_ms = 0.0;
  const bool solve = bpn > d.tol * bnorm;
  if (solve) {
    sem_solve_desc din = d;
    din.tol = d.tol * bnorm / bpn;
    status = din.solver == SEM_SOLVER_FGMRES
                 ? run_fgmres(M, P, Q->bp.p, Q->dx.p, din, info, st, true, false)
                 : run_solve(M, P, Q->bp.p, Q->dx.p, din, info, st, true, false);
    const double one = 1.0;
    launch_combine(n, Q->dx.p, ws, 1, &one, x, st);
  }
  info.bnorm = bnorm;
  info.res0 = bpn;
  info.status = status;
  if (solve && status != SEM_ENUMERIC && status != SEM_ETIMEOUT) {
    // grow the basis with dx (or restart it from x once it is full); not
    // with the results of a solve whose kernels left work undone
    const double *v = Q->dx.p;
    if (Q->nvec == Q->Lmax) {
      Q->nvec = 0;
      v = x;
    }
    const int kk = Q->nvec;
    double *Av = APv + (size_t)kk * ws, *pk = Pv + (size_t)kk * ws;
    apply_assembled<double>(L, v, Av, st);
    launch_multi_dot(t, M->kred, v, APv, ws, kk + 1, c, st);
    std::vector<double> al = read_coef(kk + 1);
    double nrm2 = al[kk];
    for (int i = 0; i < kk; ++i) nrm2 -= al[i] * al[i];
    if (nrm2 > 1e-24 * al[kk] && nrm2 > 0.0) {
      std::vector<double> neg(kk + 1);
      for (int i = 0; i < kk; ++i) neg[i] = -al[i];
      SEM_CHECK_CUDA(cudaMemcpyAsync(pk, v, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      launch_combine(n, Pv, ws, kk, neg.data(), pk, st);
      launch_combine(n, APv, ws, kk, neg.data(), Av, st);
      const double s = 1.0 / std::sqrt(nrm2);
      launch_scale(n, s, pk, st);
      launch_scale(n, s, Av, st);
      Q->nvec = kk + 1;
    }
  }
  SEM_CHECK_CUDA(cudaStreamSynchronize(st));
  return status;
}

}  // namespace sem

using namespace sem;

static cudaStream_t as_stream(void *s) { return (cudaStream_t)s; }

extern "C" {

const char *sem_last_error(void) { return g_error.c_str(); }

sem_status sem_mesh_create(const sem_mesh_desc *desc, void *stream, sem_mesh **out) {
  return guarded([&] {
    SEM_REQUIRE(desc != nullptr && out != nullptr, "null desc or out");
    *out = nullptr;
    SEM_REQUIRE(desc->ex >= 1 && desc->ey >= 1 && desc->ez >= 1,
                "element counts must be >= 1");
    SEM_REQUIRE((int64_t)desc->ex * desc->ey * desc->ez <= (1ll << 31),
                "too many elements");
    std::vector<double> verts;
    const double *v = desc->verts;
    if (!v) {
      SEM_REQUIRE(desc->jitter >= 0.0 && desc->jitter < 0.5, "jitter must be in [0, 0.5)");
      verts = builtin_vertices(desc->ex, desc->ey, desc->ez, desc->jitter, desc->seed);
      v = verts.data();
    }
    std::unique_ptr<sem_mesh> M(new sem_mesh());
    cudaStream_t st = as_stream(stream);
    M->stream = st;
    build_level(M->fine, desc->ex, desc->ey, desc->ez, desc->N, desc->bc, desc->geom,
                desc->f64_arith, v, false, st);
    M->red.init(kVecMaxBlocks, 4);
    M->scal.alloc(16);
    SEM_CHECK_CUDA(cudaMemsetAsync(M->scal.p, 0, 16 * sizeof(double), st));
    SEM_CHECK_CUDA(cudaMallocHost(&M->pinned, 16 * sizeof(double)));
    SEM_CHECK_CUDA(cudaStreamSynchronize(st));
    *out = M.release();
  });
}

sem_status sem_mesh_destroy(sem_mesh *mesh) {
  return guarded([&] {
    if (!mesh) return;
    if (mesh->pinned) cudaFreeHost(mesh->pinned);
    if (mesh->kpinned) cudaFreeHost(mesh->kpinned);
    if (mesh->graph) cudaGraphExecDestroy(mesh->graph);
    if (mesh->cstream) cudaStreamDestroy(mesh->cstream);
    delete mesh;
  });
}

sem_status sem_inject_alloc_failure(int32_t after) {
  return guarded([&] {
    SEM_REQUIRE(after >= 0, "after must be >= 0 (got %d)", after);
    g_alloc_fail_countdown.store(after);
  });
}

sem_status sem_inject_wait_error(sem_mesh *mesh, void *stream) {
  return guarded([&] {
    SEM_REQUIRE(mesh != nullptr && mesh->fine.err.p != nullptr, "null mesh");
    const int one = 1;
    cudaStream_t st = as_stream(stream);
    SEM_CHECK_CUDA(cudaMemcpyAsync(mesh->fine.err.p, &one, sizeof(int), cudaMemcpyHostToDevice,
                                   st));
    SEM_CHECK_CUDA(cudaStreamSynchronize(st));
  });
}

sem_status sem_mesh_info(const sem_mesh *mesh, int64_t *n_local, int64_t *n_global,
                         size_t *dev_bytes) {
  return guarded([&] {
    SEM_REQUIRE(mesh != nullptr, "null mesh");
    if (n_local) *n_local = mesh->fine.t.nl;
    if (n_global) *n_global = mesh->fine.t.ng;
    if (dev_bytes)
      *dev_bytes = mesh->fine.device_bytes() + mesh->work.bytes() + mesh->red.partials.bytes() +
                   mesh->krylov.bytes() + mesh->kred.partials.bytes() + mesh->kscal.bytes() +
                   mesh->scal.bytes() + mesh->host_b.bytes() + mesh->host_x.bytes();
  });
}

sem_status sem_mesh_field(sem_mesh *mesh, int32_t which, double *out, void *stream) {
  return guarded([&] {
    SEM_REQUIRE(mesh != nullptr && out != nullptr, "null mesh or output");
    SEM_REQUIRE(which >= SEM_FIELD_X && which <= SEM_FIELD_DINV, "unknown field %d", which);
    launch_field(mesh->fine, which, out, as_stream(stream));
  });
}

sem_status sem_ax(sem_mesh *mesh, sem_dtype dtype, const void *u, void *w, int32_t flags,
                  void *stream) {
  return guarded([&] {
    SEM_REQUIRE(mesh != nullptr && u != nullptr && w != nullptr, "null mesh or vector");
    SEM_REQUIRE(u != w, "u and w must not alias");
    SEM_REQUIRE(flags == SEM_AX_LOCAL || flags == SEM_AX_ASSEMBLED, "unknown flags %d", flags);
    cudaStream_t st = as_stream(stream);
    if (dtype == SEM_F64) {
      launch_ax<double>(mesh->fine, (const double *)u, (double *)w, st);
      if (flags == SEM_AX_ASSEMBLED) {
        launch_gs<double>(mesh->fine, (double *)w, st);
        launch_mask<double>(mesh->fine, (double *)w, st);
      }
    } else if (dtype == SEM_F32 && mesh->fine.geom != SEM_GEOM_STORED) {
      if (!mesh->fine.dinv32.p) level_ensure_f32(mesh->fine, st);
      launch_ax<float>(mesh->fine, (const float *)u, (float *)w, st);
      if (flags == SEM_AX_ASSEMBLED) {
        launch_gs<float>(mesh->fine, (float *)w, st);
        launch_mask<float>(mesh->fine, (float *)w, st);
      }
    } else if (dtype == SEM_F32 || dtype == SEM_F16 || dtype == SEM_BF16) {
      if (dtype == SEM_F32) {
        if (!mesh->fine.G32.p) level_ensure_f32(mesh->fine, st);
      } else {
        level_ensure_g16(mesh->fine, dtype, st);
      }
      launch_ax32(mesh->fine, dtype, (const float *)u, (float *)w, flags == SEM_AX_ASSEMBLED, st);
      // the staged kernel leaves its work undone if a bounded wait ran out
      if (take_wait_errors(mesh, nullptr, st))
        fail(SEM_ETIMEOUT, "a bounded wait in the operator kernel ran out (a bulk copy did not "
                           "complete); w is incomplete");
    } else {
      fail(SEM_EINVAL, "unknown dtype %d", (int)dtype);
    }
  });
}

sem_status sem_gs(sem_mesh *mesh, sem_dtype dtype, void *u, void *stream) {
  return guarded([&] {
    SEM_REQUIRE(mesh != nullptr && u != nullptr, "null mesh or vector");
    SEM_REQUIRE(dtype == SEM_F64 || dtype == SEM_F32, "sem_gs supports SEM_F64 and SEM_F32");
    const Level &L = mesh->fine;
    cudaStream_t st = as_stream(stream);
    // the face-plane passes (every copy gets the same bits) where the plane
    // indices fit 32 bits, else the per-node table
    const bool planes = (uint64_t)L.t.E * L.t.Np * L.t.Np < (1ull << 32);
    if (dtype == SEM_F64) {
      if (planes) launch_planes_assemble<double>(L, (double *)u, st, false);
      else launch_gs<double>(L, (double *)u, st);
    } else {
      if (planes) launch_planes_assemble<float>(L, (float *)u, st, false);
      else launch_gs<float>(L, (float *)u, st);
    }
  });
}

sem_status sem_dot(sem_mesh *mesh, const double *u, const double *v, double *result,
                   void *stream) {
  return guarded([&] {
    SEM_REQUIRE(mesh && u && v && result, "null argument");
    cudaStream_t st = as_stream(stream);
    launch_dot(mesh->fine.t, mesh->red, u, v, mesh->scal.p + 15, st);
    SEM_CHECK_CUDA(cudaMemcpyAsync(result, mesh->scal.p + 15, sizeof(double),
                                   cudaMemcpyDeviceToHost, st));
    SEM_CHECK_CUDA(cudaStreamSynchronize(st));
  });
}

sem_status sem_pmg_setup(sem_mesh *mesh, const sem_pmg_desc *desc, void *stream, sem_pmg **out) {
  return guarded([&] {
    SEM_REQUIRE(mesh && desc && out, "null argument");
    *out = nullptr;
    std::unique_ptr<sem_pmg> P(new sem_pmg());
    static std::atomic<uint64_t> serials{0};
    P->serial = ++serials;
    pmg_build(P.get(), mesh, *desc, as_stream(stream));
    *out = P.release();
  });
}

sem_status sem_pmg_destroy(sem_pmg *pmg) {
  return guarded([&] { delete pmg; });
}

sem_status sem_pmg_coarse_iters(const sem_pmg *pmg, void *stream, int32_t *iters) {
  return guarded([&] {
    SEM_REQUIRE(pmg != nullptr && iters != nullptr, "null argument");
    *iters = 0;
    if (!pmg->persistent_coarse || !pmg->coarse.iters.p) return;
    int v = 0;
    SEM_CHECK_CUDA(cudaMemcpyAsync(&v, pmg->coarse.iters.p, sizeof(int), cudaMemcpyDeviceToHost,
                                   as_stream(stream)));
    SEM_CHECK_CUDA(cudaStreamSynchronize(as_stream(stream)));
    *iters = v;
  });
}

sem_status sem_pmg_coarse_solve(sem_pmg *pmg, const double *b, double *x, void *stream) {
  return guarded([&] {
    SEM_REQUIRE(pmg && b && x, "null argument");
    SEM_REQUIRE(b != x, "b and x must not alias");
    pmg_coarse_solve(pmg, b, x, as_stream(stream));
  });
}

sem_status sem_pmg_info(const sem_pmg *pmg, int32_t level, double *lam_lo, double *lam_hi) {
  return guarded([&] {
    SEM_REQUIRE(pmg != nullptr, "null pmg");
    SEM_REQUIRE(level >= 0 && level < (int)pmg->levp.size(), "level %d out of range", level);
    if (lam_lo) *lam_lo = pmg->levp[level]->lam_lo;
    if (lam_hi) *lam_hi = pmg->levp[level]->lam_hi;
  });
}

sem_status sem_pmg_vcycle(sem_pmg *pmg, const double *r, double *z, void *stream) {
  return guarded([&] {
    SEM_REQUIRE(pmg && r && z, "null argument");
    SEM_REQUIRE(r != z, "r and z must not alias");
    cudaStream_t st = as_stream(stream);
    pmg_vcycle(pmg, r, z, st);
    // staged smoother kernels leave their work undone if a bounded wait ran out
    if (take_wait_errors(pmg->mesh, pmg, st))
      fail(SEM_ETIMEOUT, "a bounded wait in a smoother kernel ran out (a bulk copy did not "
                         "complete); z is incomplete");
  });
}

static void check_solve_args(sem_mesh *mesh, sem_pmg *pmg, const sem_solve_desc *desc,
                             sem_solve_info *info) {
  SEM_REQUIRE(mesh && desc && info, "null argument");
  SEM_REQUIRE(desc->solver == SEM_SOLVER_PCG || desc->solver == SEM_SOLVER_FLEXCG ||
                  desc->solver == SEM_SOLVER_FGMRES,
              "unknown solver %d", desc->solver);
  SEM_REQUIRE(desc->solver != SEM_SOLVER_FLEXCG || pmg != nullptr,
              "SEM_SOLVER_FLEXCG needs a pMG preconditioner");
  SEM_REQUIRE(desc->solver != SEM_SOLVER_FGMRES ||
                  (desc->restart >= 0 && desc->restart <= kMaxKrylov),
              "restart %d outside [0, %d]", desc->restart, kMaxKrylov);
  SEM_REQUIRE(pmg == nullptr || pmg->mesh == mesh, "pmg was built on another mesh");
  SEM_REQUIRE(desc->tol >= 0.0 && desc->max_iter >= 0, "negative tol or max_iter");
  SEM_REQUIRE(desc->use_graph == 0 || desc->use_graph == 1, "use_graph must be 0 or 1");
  SEM_REQUIRE(desc->zero_guess == 0 || desc->zero_guess == 1, "zero_guess must be 0 or 1");
  SEM_REQUIRE(desc->use_graph == 0 || desc->solver == SEM_SOLVER_FLEXCG,
              "use_graph applies to SEM_SOLVER_FLEXCG only");
}

sem_status sem_solve(sem_mesh *mesh, sem_pmg *pmg, const double *b, double *x,
                     const sem_solve_desc *desc, sem_solve_info *info, void *stream) {
  sem_status result = SEM_OK;
  sem_status st = guarded([&] {
    check_solve_args(mesh, pmg, desc, info);
    SEM_REQUIRE(b && x && b != (const double *)x, "null or aliased b and x");
    std::memset(info, 0, sizeof(*info));
    result = desc->solver == SEM_SOLVER_FGMRES
                 ? run_fgmres(mesh, pmg, b, x, *desc, *info, as_stream(stream))
                 : run_solve(mesh, pmg, b, x, *desc, *info, as_stream(stream));
  });
  return st != SEM_OK ? st : result;
}

sem_status sem_solve_host(sem_mesh *mesh, sem_pmg *pmg, const double *b_host, double *x_host,
                          const sem_solve_desc *desc, sem_solve_info *info, void *stream) {
  sem_status result = SEM_OK;
  sem_status st = guarded([&] {
    check_solve_args(mesh, pmg, desc, info);
    SEM_REQUIRE(b_host && x_host, "null host vector");
    std::memset(info, 0, sizeof(*info));
    const size_t n = (size_t)mesh->fine.t.nl;
    if (!mesh->host_b.p) {
      mesh->host_b.alloc(n);
      mesh->host_x.alloc(n);
    }
    cudaStream_t s = as_stream(stream);
    SEM_CHECK_CUDA(cudaMemcpyAsync(mesh->host_b.p, b_host, n * sizeof(double),
                                   cudaMemcpyHostToDevice, s));
    if (!desc->zero_guess)
      SEM_CHECK_CUDA(cudaMemcpyAsync(mesh->host_x.p, x_host, n * sizeof(double),
                                     cudaMemcpyHostToDevice, s));
    result = desc->solver == SEM_SOLVER_FGMRES
                 ? run_fgmres(mesh, pmg, mesh->host_b.p, mesh->host_x.p, *desc, *info, s)
                 : run_solve(mesh, pmg, mesh->host_b.p, mesh->host_x.p, *desc, *info, s);
    SEM_CHECK_CUDA(cudaMemcpyAsync(x_host, mesh->host_x.p, n * sizeof(double),
                                   cudaMemcpyDeviceToHost, s));
    SEM_CHECK_CUDA(cudaStreamSynchronize(s));
  });
  return st != SEM_OK ? st : result;
}

sem_status sem_proj_create(sem_mesh *mesh, int32_t Lmax, void *stream, sem_proj **out) {
  return guarded([&] {
    SEM_REQUIRE(mesh != nullptr && out != nullptr, "null mesh or out");
    SEM_REQUIRE(Lmax >= 1 && Lmax <= kMaxKrylov - 1, "Lmax %d outside [1, %d]", Lmax,
                kMaxKrylov - 1);
    *out = nullptr;
    std::unique_ptr<sem_proj> Q(new sem_proj());
    Q->mesh = mesh;
    Q->Lmax = Lmax;
    const size_t ws = work_stride(mesh);
    Q->P.alloc((size_t)Lmax * ws);
    Q->AP.alloc((size_t)(Lmax + 1) * ws);
    Q->bp.alloc(ws);
    Q->dx.alloc(ws);
    Q->coef.alloc(kMaxKrylov + 2);
    SEM_CHECK_CUDA(cudaStreamSynchronize(as_stream(stream)));
    *out = Q.release();
  });
}

sem_status sem_proj_destroy(sem_proj *proj) {
  return guarded([&] { delete proj; });
}

sem_status sem_proj_info(const sem_proj *proj, int32_t *nvec) {
  return guarded([&] {
    SEM_REQUIRE(proj != nullptr && nvec != nullptr, "null argument");
    *nvec = proj->nvec;
  });
}

sem_status sem_solve_projected(sem_mesh *mesh, sem_pmg *pmg, sem_proj *proj, const double *b,
                               double *x, const sem_solve_desc *desc, sem_solve_info *info,
                               void *stream) {
  sem_status result = SEM_OK;
  sem_status st = guarded([&] {
    check_solve_args(mesh, pmg, desc, info);
    SEM_REQUIRE(proj != nullptr && proj->mesh == mesh, "projection handle of another mesh");
    SEM_REQUIRE(b && x && b != (const double *)x, "null or aliased b and x");
    std::memset(info, 0, sizeof(*info));
    cudaStream_t s = as_stream(stream);
    cudaEvent_t e0, e1;
    SEM_CHECK_CUDA(cudaEventCreate(&e0));
    SEM_CHECK_CUDA(cudaEventCreate(&e1));
    SEM_CHECK_CUDA(cudaEventRecord(e0, s));
    result = run_projected(mesh, pmg, proj, b, x, *desc, *info, s);
    SEM_CHECK_CUDA(cudaEventRecord(e1, s));
    SEM_CHECK_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    info->time_ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  });
  return st != SEM_OK ? st : result;
}

}  // extern "C"
