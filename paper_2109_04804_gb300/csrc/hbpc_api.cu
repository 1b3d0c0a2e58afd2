// C-ABI of libhbpc (include/hbpc.h): context set-up, the Newton-GMRES stage
// solve (Sec. 3.2, 4.2) and the HBPC(q, k_max) driver (Algorithm 1, Sec. 2.1).
// The host only sequences launches; every vector of the method lives on the
// device and the per-iteration GMRES state is device-resident, so the host
// waits on the GPU once per batch of GMRES iterations and once per Newton
// iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/hbpc.h"
#include "dg_ops.cuh"
#include "hbpc_internal.h"
#include "krylov.cuh"
#include "bjext_kernels.cuh"

namespace hbpc {

// ---------------------------------------------------------------------------
// small vector kernels
// ---------------------------------------------------------------------------
constexpr int kMaxTerms = 12;
struct LinComb {
  const double* x[kMaxTerms];
  double c[kMaxTerms];
  int nterm;
};

// out = sum_t c_t x_t  (grid-stride)
__global__ void k_lincomb(LinComb lc, double* out, size_t n) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    double a = 0.0;
    for (int t = 0; t < lc.nterm; ++t) a += lc.c[t] * lc.x[t][i];
    out[i] = a;
  }
}

// y += x
__global__ void k_add(const double* x, double* y, size_t n) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x)
    y[i] += x[i];
}

// out = -a - b
__global__ void k_neg_sum(const double* a, const double* b, double* out, size_t n) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x)
    out[i] = -a[i] - b[i];
}

__global__ void k_set2(double* p, double a, double b) {
  if (threadIdx.x == 0) { p[0] = a; p[1] = b; }
}

// sqrt of the three squared norms in st->nrm into out[0..2]
__global__ void k_sqrt_norms(const GmresState* st, double* out) {
  if (threadIdx.x < 3) out[threadIdx.x] = sqrt(st->nrm[threadIdx.x]);
}

}  // namespace hbpc

using namespace hbpc;

static thread_local std::string g_create_error;

namespace {
// Per-launch device timing with CUDA events (enabled by hbpc_profile_enable).
struct Prof {
  bool on = false;
  double ms[HBPC_NPHASES] = {};
  long long cnt[HBPC_NPHASES] = {};
  struct Pend { int ph; cudaEvent_t a, b; };
  std::vector<cudaEvent_t> pool;
  std::vector<Pend> pend;
  cudaEvent_t get() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
};
}  // namespace

struct hbpc_ctx {
  hbpc_mesh mesh{};
  hbpc_physics phys{};
  hbpc_solver sol{};
  int N = 0, P = 0, nodes = 0, dim = 0, nv = 0;
  long long nE = 0, ndof = 0;
  cudaStream_t stream = nullptr;
  OpsTable ops;
  DGParams<double> prm{};
  Basis1D basis;
  // tableau
  int s = 0;
  double c[4] = {0, 0, 0, 0}, B1[4][4] = {}, B2[4][4] = {};
  // device memory
  double* Wn = nullptr;     // state w^n
  double* X = nullptr;      // Newton unknown (W, S)
  double* G = nullptr;      // residual
  double* r1 = nullptr;     // R1(W) at the Newton iterate
  double* r2 = nullptr;     // R2(W, S) at the Newton iterate
  double* dX = nullptr;     // Newton increment
  double* bvec = nullptr;   // stage right-hand side
  double* stage = nullptr;  // 2 levels x s stages x (w, r1, r2)
  double* V = nullptr;      // Krylov basis (m + 1) x 2 n_dof
  double* small = nullptr;  // H, cs, sn, g, vscale, nrmW, nrmS, hc, y, c12, dxn
  double* partial = nullptr;
  unsigned* ticket = nullptr;
  GmresState* st = nullptr;
  GmresState* st_host = nullptr;   // pinned mirror
  double* c12 = nullptr;    // device c1, c2
  double* dxn = nullptr;    // device norms of dX (total, W, S)
  // BJ_ext preconditioner (Sec. 3.2.3)
  int nb = 0;               // block size n_var (N+1)^dim
  double* Jpc = nullptr;    // element Jacobians, n_E x n_b x n_b
  double* Mpc = nullptr;    // (I - c1 J + c2 J^2)^-1 per element
  double* Z = nullptr;      // preconditioned Krylov vector, 2 n_dof
  double* zn = nullptr;     // device norms of Z (total, W, S)
  int* singular = nullptr;  // device flag set by the inverse
  int pc_grid = 0, pc_threads = 0;
  size_t pc_smem = 0;
  bool pc_built = false;
  double pc_c1 = 0.0, pc_c2 = 0.0;
  Krylov K{};
  hbpc_stats stats{};
  std::string err;
  int nblocks = 0;
  int verbose = 0;          // HBPC_VERBOSE=1: Newton/GMRES trace on stderr
  Prof prof;
};

namespace {

constexpr int kMaxPcBlock = 160;   // largest BJ_ext block (shared-memory inverse)

hbpc_status fail(hbpc_ctx* ctx, hbpc_status code, const std::string& msg) {
  if (ctx) ctx->err = msg; else g_create_error = msg;
  return code;
}

hbpc_status cuda_fail(hbpc_ctx* ctx, cudaError_t e, const char* where) {
  return fail(ctx, HBPC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define HBPC_CK(ctx, call)                                          \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);      \
  } while (0)

#define HBPC_LAUNCH_CK(ctx, what)                                   \
  do {                                                              \
    cudaError_t e_ = cudaGetLastError();                            \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, what);       \
  } while (0)

struct ProfTok { cudaEvent_t a = nullptr; };

ProfTok prof_begin(hbpc_ctx* x) {
  ProfTok t;
  if (x->prof.on) {
    t.a = x->prof.get();
    cudaEventRecord(t.a, x->stream);
  }
  return t;
}

void prof_end(hbpc_ctx* x, int ph, ProfTok t) {
  if (!x->prof.on || !t.a) return;
  cudaEvent_t b = x->prof.get();
  cudaEventRecord(b, x->stream);
  x->prof.pend.push_back({ph, t.a, b});
}

void prof_flush(hbpc_ctx* x) {
  for (auto& p : x->prof.pend) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      x->prof.ms[p.ph] += ms;
      x->prof.cnt[p.ph] += 1;
    }
    x->prof.pool.push_back(p.a);
    x->prof.pool.push_back(p.b);
  }
  x->prof.pend.clear();
}

// Launch statement(s) `...` counted as `n` kernel launches of phase `ph`.
#define HBPC_RUN(x, ph, n, ...)                   \
  do {                                            \
    ProfTok tok_ = prof_begin(x);                 \
    __VA_ARGS__;                                  \
    prof_end(x, ph, tok_);                        \
    (x)->stats.launches += (n);                   \
  } while (0)

void tableau(int q, hbpc_ctx* x) {
  // Appendix A, Eq. A.1-A.3
  std::memset(x->B1, 0, sizeof(x->B1));
  std::memset(x->B2, 0, sizeof(x->B2));
  if (q == 4) {
    x->s = 2;
    x->c[0] = 0; x->c[1] = 1;
    x->B1[1][0] = 0.5; x->B1[1][1] = 0.5;
    x->B2[1][0] = 1.0 / 12; x->B2[1][1] = -1.0 / 12;
  } else if (q == 6) {
    x->s = 3;
    x->c[0] = 0; x->c[1] = 0.5; x->c[2] = 1;
    const double b1[2][3] = {{101.0 / 480, 8.0 / 30, 55.0 / 2400}, {7.0 / 30, 16.0 / 30, 7.0 / 30}};
    const double b2[2][3] = {{65.0 / 4800, -25.0 / 600, -25.0 / 8000}, {5.0 / 300, 0.0, -5.0 / 300}};
    for (int l = 0; l < 2; ++l)
      for (int j = 0; j < 3; ++j) { x->B1[l + 1][j] = b1[l][j]; x->B2[l + 1][j] = b2[l][j]; }
  } else {
    x->s = 4;
    x->c[0] = 0; x->c[1] = 1.0 / 3; x->c[2] = 2.0 / 3; x->c[3] = 1;
    const double b1[3][4] = {{6893.0 / 54432, 313.0 / 2016, 89.0 / 2016, 397.0 / 54432},
                             {223.0 / 1701, 20.0 / 63, 13.0 / 63, 20.0 / 1701},
                             {31.0 / 224, 81.0 / 224, 81.0 / 224, 31.0 / 224}};
    const double b2[3][4] = {{1283.0 / 272160, -851.0 / 30240, -269.0 / 30240, -163.0 / 272160},
                             {43.0 / 8505, -16.0 / 945, -19.0 / 945, -8.0 / 8505},
                             {19.0 / 3360, -9.0 / 1120, 9.0 / 1120, -19.0 / 3360}};
    for (int l = 0; l < 3; ++l)
      for (int j = 0; j < 4; ++j) { x->B1[l + 1][j] = b1[l][j]; x->B2[l + 1][j] = b2[l][j]; }
  }
}

int grid_for(size_t n) {
  size_t g = (n + 255) / 256;
  return int(std::min<size_t>(g, 152 * 8));
}

hbpc_status lincomb(hbpc_ctx* x, double* out, std::initializer_list<std::pair<double, const double*>> terms) {
  LinComb lc{};
  for (auto& t : terms) {
    if (t.first == 0.0) continue;
    lc.x[lc.nterm] = t.second;
    lc.c[lc.nterm] = t.first;
    ++lc.nterm;
  }
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_lincomb<<<grid_for(x->ndof), 256, 0, x->stream>>>(lc, out, size_t(x->ndof)));
  HBPC_LAUNCH_CK(x, "k_lincomb");
  return HBPC_OK;
}

hbpc_status sync(hbpc_ctx* x, const char* where) {
  cudaError_t e = cudaStreamSynchronize(x->stream);
  if (e != cudaSuccess) return cuda_fail(x, e, where);
  if (x->prof.on) prof_flush(x);
  return HBPC_OK;
}

hbpc_status read_state(hbpc_ctx* x) {
  HBPC_CK(x, cudaMemcpyAsync(x->st_host, x->st, sizeof(GmresState), cudaMemcpyDeviceToHost, x->stream));
  return sync(x, "read GMRES state");
}

// squared norms of a 2 n_dof vector into st->nrm (and sqrt into out3 if given)
hbpc_status norms(hbpc_ctx* x, const double* v, size_t n, double* out3 = nullptr) {
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_norms<<<x->nblocks, kVecThreads, 0, x->stream>>>(v, n, size_t(x->ndof), x->K, nullptr));
  HBPC_LAUNCH_CK(x, "k_norms");
  if (out3) {
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_sqrt_norms<<<1, 32, 0, x->stream>>>(x->st, out3));
    HBPC_LAUNCH_CK(x, "k_sqrt_norms");
  }
  return HBPC_OK;
}

JvCoef jv_coef(hbpc_ctx* x) {
  JvCoef c;
  c.c1 = x->c12;
  c.c2 = x->c12 + 1;
  c.sqrt_eps_machine = std::sqrt(std::ldexp(1.0, -52));
  c.eps_ref = x->phys.eps;
  return c;
}

// q = J z  for the input described by z (Eq. 23 / Eq. 24)
hbpc_status apply_jv(hbpc_ctx* x, const JvInput& z) {
  const double* W = x->X;
  const double* S = x->X + x->ndof;
  if (x->ops.jv_linear) {
    HBPC_RUN(x, HBPC_PHASE_JV, 1, x->ops.jv_linear(x->prm, z, jv_coef(x), x->stream));
  } else {
    HBPC_RUN(x, HBPC_PHASE_JV, 2, x->ops.jv_fd(x->prm, W, S, x->r1, x->r2, z, jv_coef(x), x->stream));
  }
  HBPC_LAUNCH_CK(x, "jv");
  return HBPC_OK;
}

JvInput krylov_input(hbpc_ctx* x) {
  JvInput z{};
  z.V = x->V; z.ld = size_t(2 * x->ndof); z.half = size_t(x->ndof);
  z.jidx = &x->st->j;
  z.vscale = x->K.vscale;
  z.nrmW = x->K.nrmW; z.nrmS = x->K.nrmS;
  z.skip = &x->st->done;
  z.out = x->V; z.out_ld = size_t(2 * x->ndof); z.out_offset = 1;
  z.out_jidx = &x->st->j;
  if (x->sol.pc == HBPC_PC_BJEXT) {   // Jv acts on z = P^-1 v_j, kept in Z
    z.V = x->Z; z.jidx = nullptr; z.vscale = nullptr;
    z.nrmW = x->zn + 1; z.nrmS = x->zn + 2;
  }
  return z;
}

// P^-1 applied to scale * in -> out (out += when accumulate), norms to x->zn
hbpc_status pc_apply(hbpc_ctx* x, const double* in, const int* jidx, const double* scale,
                     double* out, int accumulate, const int* skip) {
  PcApply a{};
  a.M = x->Mpc; a.J = x->Jpc;
  a.xW = in; a.xS = in + x->ndof;
  a.scale = scale; a.jidx = jidx; a.ld = size_t(2 * x->ndof);
  a.oW = out; a.oS = out + x->ndof;
  a.c12 = x->c12; a.skip = skip; a.accumulate = accumulate; a.zn = x->zn;
  a.nb = x->nb; a.nE = int(x->nE);
  HBPC_RUN(x, HBPC_PHASE_PC, 1, k_pc_apply<<<x->pc_grid, x->pc_threads, x->pc_smem, x->stream>>>(a, x->K));
  HBPC_LAUNCH_CK(x, "k_pc_apply");
  return HBPC_OK;
}

// Build J_i, S_i and M_i = S_i^-1 at the state W for the current c1, c2.
hbpc_status pc_build(hbpc_ctx* x, const double* W, double c1, double c2) {
  const bool linear = x->phys.law == HBPC_LAW_ADVECTION;
  if (linear && x->pc_built && x->pc_c1 == c1 && x->pc_c2 == c2) return HBPC_OK;
  const size_t nb = size_t(x->nb);
  HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1, x->ops.pc_assemble(x->prm, W, x->Jpc, x->stream));
  HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1,
           k_pc_form_S<<<int(x->nE), 256, nb * nb * sizeof(double), x->stream>>>(x->Jpc, x->Mpc, x->nb,
                                                                                   int(x->nE), x->c12));
  HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1,
           k_pc_invert<<<int(x->nE), 256, (nb * nb + nb) * sizeof(double) + nb * sizeof(int), x->stream>>>(
               x->Mpc, x->nb, int(x->nE), x->singular));
  HBPC_LAUNCH_CK(x, "pc build");
  int sing = 0;
  HBPC_CK(x, cudaMemcpyAsync(&sing, x->singular, sizeof(int), cudaMemcpyDeviceToHost, x->stream));
  hbpc_status s = sync(x, "pc build");
  if (s != HBPC_OK) return s;
  if (sing) return fail(x, HBPC_ERR_NONFINITE, "BJ_ext block is singular");
  x->pc_built = true;
  x->pc_c1 = c1;
  x->pc_c2 = c2;
  return HBPC_OK;
}

hbpc_status arnoldi_step(hbpc_ctx* x) {
  hbpc_status s;
  if (x->sol.pc == HBPC_PC_BJEXT) {
    s = pc_apply(x, x->V, &x->st->j, x->K.vscale, x->Z, 0, &x->st->done);
    if (s != HBPC_OK) return s;
  }
  s = apply_jv(x, krylov_input(x));
  if (s != HBPC_OK) return s;
  const size_t sm = sizeof(double) * size_t(x->K.m + 3);
  HBPC_RUN(x, HBPC_PHASE_DOT, 1, k_arnoldi_dot<<<x->nblocks, kVecThreads, sm, x->stream>>>(x->K, 0));
  HBPC_RUN(x, HBPC_PHASE_UPDATE, 1, k_arnoldi_update<<<x->nblocks, kVecThreads, sm, x->stream>>>(x->K, 0));
  HBPC_RUN(x, HBPC_PHASE_DOT, 1, k_arnoldi_dot<<<x->nblocks, kVecThreads, sm, x->stream>>>(x->K, 1));
  HBPC_RUN(x, HBPC_PHASE_UPDATE, 1, k_arnoldi_update<<<x->nblocks, kVecThreads, sm, x->stream>>>(x->K, 1));
  HBPC_LAUNCH_CK(x, "arnoldi");
  return HBPC_OK;
}

// Solve J dX = -G (G in x->G with squared norms in st->nrm) by restarted GMRES
// from dX = 0; returns the iteration count through *its.
hbpc_status gmres(hbpc_ctx* x, int* its_out, bool* conv_out) {
  const size_t n2 = size_t(2 * x->ndof);
  HBPC_CK(x, cudaMemsetAsync(x->dX, 0, n2 * sizeof(double), x->stream));
  HBPC_CK(x, cudaMemcpyAsync(x->V, x->G, n2 * sizeof(double), cudaMemcpyDeviceToDevice, x->stream));
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_cycle_init<<<1, 32, 0, x->stream>>>(x->K, -1.0, x->sol.tol_gmres_rel, 1, x->sol.gmres_max_iter));
  HBPC_LAUNCH_CK(x, "k_cycle_init");
  const int batch = 4;
  for (;;) {
    for (int b = 0; b < batch; ++b) {
      hbpc_status s = arnoldi_step(x);
      if (s != HBPC_OK) return s;
    }
    hbpc_status s = read_state(x);
    if (s != HBPC_OK) return s;
    const GmresState& h = *x->st_host;
    if (!(h.resid == h.resid) || std::isinf(h.resid))
      return fail(x, HBPC_ERR_NONFINITE, "GMRES residual is not finite");
    if (!h.done) continue;
    // end of a cycle: dX += V y
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_solve_y<<<1, 32, 0, x->stream>>>(x->K));
    if (x->sol.pc == HBPC_PC_BJEXT) {   // dX += P^-1 (V y)
      HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_combine<<<x->nblocks, kVecThreads, sizeof(double) * size_t(x->K.m + 1), x->stream>>>(x->K, x->Z, 0));
      s = pc_apply(x, x->Z, nullptr, nullptr, x->dX, 1, nullptr);
      if (s != HBPC_OK) return s;
    } else {
      HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_combine<<<x->nblocks, kVecThreads, sizeof(double) * size_t(x->K.m + 1), x->stream>>>(x->K, x->dX, 1));
    }
    HBPC_LAUNCH_CK(x, "gmres update");
    if (h.converged || h.its >= h.max_its) {
      *its_out = h.its;
      *conv_out = h.converged != 0;
      return HBPC_OK;
    }
    // restart: V_0 = -G - J dX
    s = norms(x, x->dX, n2, x->dxn);
    if (s != HBPC_OK) return s;
    JvInput z{};
    z.V = x->dX; z.ld = n2; z.half = size_t(x->ndof);
    z.jidx = nullptr; z.vscale = nullptr;
    z.nrmW = x->dxn + 1; z.nrmS = x->dxn + 2;
    z.skip = nullptr;
    z.out = x->V + n2; z.out_ld = n2; z.out_offset = 0; z.out_jidx = nullptr;
    s = apply_jv(x, z);
    if (s != HBPC_OK) return s;
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_neg_sum<<<grid_for(n2), 256, 0, x->stream>>>(x->G, x->V + n2, x->V, n2));
    s = norms(x, x->V, n2);
    if (s != HBPC_OK) return s;
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_cycle_init<<<1, 32, 0, x->stream>>>(x->K, 1.0, x->sol.tol_gmres_rel, 0, x->sol.gmres_max_iter));
    HBPC_LAUNCH_CK(x, "k_cycle_init");
  }
}

hbpc_status residual(hbpc_ctx* x, const double* b, double c1, double c2) {
  const long long n = x->ndof;
  HBPC_RUN(x, HBPC_PHASE_OPERATOR, 1,
           x->ops.residual(x->prm, x->X, x->X + n, b, c1, c2, x->G, x->G + n, x->r1, x->r2, x->stream));
  HBPC_LAUNCH_CK(x, "residual");
  x->stats.r1_evals += 1;
  x->stats.r2_evals += 1;
  return norms(x, x->G, size_t(2 * n));
}

// Newton on G(X) = 0 from X^0 = (W0, R1(W0)).  Result in x->X.
hbpc_status newton(hbpc_ctx* x, const double* b, double a1, double a2, const double* W0) {
  const long long n = x->ndof;
  const double dt = x->sol.dt;
  const double c1 = a1 * dt, c2 = a2 * dt * dt / 2.0;
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_set2<<<1, 32, 0, x->stream>>>(x->c12, c1, c2));
  if (W0 != x->X) HBPC_CK(x, cudaMemcpyAsync(x->X, W0, n * sizeof(double), cudaMemcpyDeviceToDevice, x->stream));
  HBPC_RUN(x, HBPC_PHASE_OPERATOR, 1, x->ops.r1(x->prm, x->X, x->X + n, x->stream));
  HBPC_LAUNCH_CK(x, "r1");
  x->stats.r1_evals += 1;
  hbpc_status s = residual(x, b, c1, c2);
  if (s != HBPC_OK) return s;
  if ((s = read_state(x)) != HBPC_OK) return s;
  const double g0 = std::sqrt(x->st_host->nrm[0]);
  if (!std::isfinite(g0)) return fail(x, HBPC_ERR_NONFINITE, "initial Newton residual is not finite");
  x->stats.newton_solves += 1;
  if (x->verbose) std::fprintf(stderr, "[hbpc] newton a1=%g a2=%g ||G0||=%.6e\n", a1, a2, g0);
  if (g0 == 0.0) return HBPC_OK;
  for (int r = 0; r < x->sol.newton_max_iter; ++r) {
    int its = 0;
    bool conv = false;
    if (x->sol.pc == HBPC_PC_BJEXT && (s = pc_build(x, x->X, c1, c2)) != HBPC_OK) return s;
    if ((s = gmres(x, &its, &conv)) != HBPC_OK) return s;
    x->stats.gmres_its += its;
    x->stats.newton_its += 1;
    const int per = x->ops.jv_linear ? 2 : 3;
    x->stats.r1_evals += (long long)its * (x->ops.jv_linear ? 2 : 1);
    x->stats.r2_evals += (long long)its * (per - (x->ops.jv_linear ? 2 : 1));
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_add<<<grid_for(size_t(2 * n)), 256, 0, x->stream>>>(x->dX, x->X, size_t(2 * n)));
    HBPC_LAUNCH_CK(x, "newton update");
    if ((s = norms(x, x->dX, size_t(2 * n))) != HBPC_OK) return s;
    if ((s = read_state(x)) != HBPC_OK) return s;
    const double dW = std::sqrt(x->st_host->nrm[1]);
    if ((s = residual(x, b, c1, c2)) != HBPC_OK) return s;
    if ((s = read_state(x)) != HBPC_OK) return s;
    const double gn = std::sqrt(x->st_host->nrm[0]);
    if (x->verbose)
      std::fprintf(stderr, "[hbpc]   it %d gmres %d conv %d ||G||=%.6e rel %.3e ||dW||=%.3e\n", r, its,
                   int(conv), gn, gn / g0, dW);
    if (!std::isfinite(gn) || !std::isfinite(dW))
      return fail(x, HBPC_ERR_NONFINITE, "Newton residual is not finite");
    if (gn <= x->sol.tol_newton_rel * g0 || dW <= x->sol.tol_newton_abs) return HBPC_OK;
  }
  return fail(x, HBPC_ERR_NO_CONVERGENCE, "Newton did not converge within newton_max_iter");
}

hbpc_status eval_r1r2(hbpc_ctx* x, const double* w, double* r1, double* r2) {
  HBPC_RUN(x, HBPC_PHASE_OPERATOR, 1, x->ops.r1(x->prm, w, r1, x->stream));
  HBPC_RUN(x, HBPC_PHASE_OPERATOR, 1, x->ops.r2(x->prm, w, r1, r2, x->stream));
  HBPC_LAUNCH_CK(x, "stage r1/r2");
  x->stats.r1_evals += 1;
  x->stats.r2_evals += 1;
  return HBPC_OK;
}

// One HBPC(q, k_max) step of Algorithm 1 on x->Wn.
hbpc_status hbpc_one_step(hbpc_ctx* x) {
  const long long n = x->ndof;
  const int s = x->s;
  const double dt = x->sol.dt;
  auto W = [&](int lvl, int l) { return x->stage + (size_t(lvl) * s * 3 + size_t(l) * 3 + 0) * n; };
  auto R1 = [&](int lvl, int l) { return x->stage + (size_t(lvl) * s * 3 + size_t(l) * 3 + 1) * n; };
  auto R2 = [&](int lvl, int l) { return x->stage + (size_t(lvl) * s * 3 + size_t(l) * 3 + 2) * n; };
  hbpc_status st;
  // stage 1 of every level is w^{n-1}; it is kept in level 0 and aliased
  HBPC_CK(x, cudaMemcpyAsync(W(0, 0), x->Wn, n * sizeof(double), cudaMemcpyDeviceToDevice, x->stream));
  if ((st = eval_r1r2(x, W(0, 0), R1(0, 0), R2(0, 0))) != HBPC_OK) return st;
  // predictor (Eq. 5 as Eq. 7/8)
  for (int l = 1; l < s; ++l) {
    const double dc = x->c[l] - x->c[l - 1];
    const double a1 = dc / 2.0, a2 = dc * dc / 6.0;
    if ((st = lincomb(x, x->bvec, {{1.0, W(0, l - 1)}, {a1 * dt, R1(0, l - 1)},
                                   {a2 * dt * dt / 2.0, R2(0, l - 1)}})) != HBPC_OK) return st;
    if ((st = newton(x, x->bvec, a1, a2, W(0, l - 1))) != HBPC_OK) return st;
    HBPC_CK(x, cudaMemcpyAsync(W(0, l), x->X, n * sizeof(double), cudaMemcpyDeviceToDevice, x->stream));
    if ((st = eval_r1r2(x, W(0, l), R1(0, l), R2(0, l))) != HBPC_OK) return st;
  }
  // corrector sweeps (Eq. 6): level cur -> level 1 - cur; stage 1 always from level 0
  int cur = 0;
  for (int k = 0; k < x->sol.kmax; ++k) {
    const int nxt = 1 - cur;
    auto Wc = [&](int l) { return l == 0 ? W(0, 0) : W(cur, l); };
    auto R1c = [&](int l) { return l == 0 ? R1(0, 0) : R1(cur, l); };
    auto R2c = [&](int l) { return l == 0 ? R2(0, 0) : R2(cur, l); };
    for (int l = 1; l < s; ++l) {
      LinComb lc{};
      auto add = [&](double c, const double* p) {
        if (c != 0.0) { lc.x[lc.nterm] = p; lc.c[lc.nterm] = c; ++lc.nterm; }
      };
      add(1.0, W(0, 0));
      add(-dt, R1c(l));
      add(dt * dt / 2.0, R2c(l));
      for (int j = 0; j < s; ++j) {
        add(dt * x->B1[l][j], R1c(j));
        add(dt * dt * x->B2[l][j], R2c(j));
      }
      HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_lincomb<<<grid_for(size_t(n)), 256, 0, x->stream>>>(lc, x->bvec, size_t(n)));
      HBPC_LAUNCH_CK(x, "corrector rhs");
      if ((st = newton(x, x->bvec, 1.0, 1.0, Wc(l))) != HBPC_OK) return st;
      HBPC_CK(x, cudaMemcpyAsync(W(nxt, l), x->X, n * sizeof(double), cudaMemcpyDeviceToDevice, x->stream));
      if ((st = eval_r1r2(x, W(nxt, l), R1(nxt, l), R2(nxt, l))) != HBPC_OK) return st;
    }
    cur = nxt;
  }
  const double* last = (s - 1 == 0) ? W(0, 0) : W(cur, s - 1);
  HBPC_CK(x, cudaMemcpyAsync(x->Wn, last, n * sizeof(double), cudaMemcpyDeviceToDevice, x->stream));
  return sync(x, "hbpc step");
}

template <typename Tp>
hbpc_status dmalloc(hbpc_ctx* x, Tp** p, size_t count) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(Tp));
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(x, HBPC_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return HBPC_OK;
}

void free_all(hbpc_ctx* x) {
  for (auto& p : x->prof.pend) { x->prof.pool.push_back(p.a); x->prof.pool.push_back(p.b); }
  for (cudaEvent_t e : x->prof.pool) cudaEventDestroy(e);
  x->prof.pool.clear();
  x->prof.pend.clear();
  cudaFree(x->Wn); cudaFree(x->X); cudaFree(x->G); cudaFree(x->r1); cudaFree(x->r2);
  cudaFree(x->dX); cudaFree(x->bvec); cudaFree(x->stage); cudaFree(x->V); cudaFree(x->small);
  cudaFree(x->partial); cudaFree(x->ticket); cudaFree(x->st);
  cudaFree(x->Jpc); cudaFree(x->Mpc); cudaFree(x->Z); cudaFree(x->singular);
  if (x->st_host) cudaFreeHost(x->st_host);
}

hbpc_status validate(const hbpc_mesh* mesh, int N, int nodes, const hbpc_physics* ph,
                     const hbpc_solver* so) {
  auto bad = [](const std::string& m) { return fail(nullptr, HBPC_ERR_INVALID_ARG, m); };
  if (!mesh || !ph || !so) return bad("null argument");
  if (mesh->dim < 1 || mesh->dim > 3) return bad("dim must be 1, 2 or 3");
  for (int m = 0; m < mesh->dim; ++m) {
    if (mesh->n[m] < 1) return bad("n[m] must be >= 1");
    if (!(mesh->hi[m] > mesh->lo[m])) return bad("hi must exceed lo");
  }
  if (N < 1 || N + 1 > kMaxP) return bad("N must satisfy 1 <= N <= 7");
  if (nodes != HBPC_NODES_LOBATTO && nodes != HBPC_NODES_GAUSS) return bad("unknown node family");
  if (ph->law < 0 || ph->law > 2) return bad("unknown law");
  if (ph->flux != HBPC_FLUX_GLOBAL_LF && ph->flux != HBPC_FLUX_RUSANOV) return bad("unknown flux");
  if (!(ph->eps > 0.0)) return bad("eps must be > 0");
  if (ph->law == HBPC_LAW_EULER && !(ph->gamma > 1.0)) return bad("gamma must be > 1");
  if (so->q != 4 && so->q != 6 && so->q != 8) return bad("q must be 4, 6 or 8");
  if (so->kmax < 0) return bad("kmax must be >= 0");
  if (!(so->dt > 0.0)) return bad("dt must be > 0");
  if (so->gmres_restart < 1 || so->gmres_restart > 1000) return bad("gmres_restart must be in 1..1000");
  if (so->gmres_max_iter < 1 || so->newton_max_iter < 1) return bad("iteration caps must be >= 1");
  if (!(so->tol_gmres_rel > 0.0) || !(so->tol_newton_rel >= 0.0) || !(so->tol_newton_abs >= 0.0))
    return bad("tolerances must be positive");
  if (so->pc != HBPC_PC_NONE && so->pc != HBPC_PC_BJEXT) return bad("unknown preconditioner");
  if (so->pc == HBPC_PC_BJEXT) {
    int nb = (ph->law == HBPC_LAW_EULER) ? mesh->dim + 2 : 1;
    for (int m = 0; m < mesh->dim; ++m) nb *= (N + 1);
    if (nb > kMaxPcBlock)
      return fail(nullptr, HBPC_ERR_UNSUPPORTED, "BJ_ext block n_var (N+1)^dim exceeds the supported size");
  }
  if (so->precision != HBPC_PREC_FP64) return fail(nullptr, HBPC_ERR_UNSUPPORTED, "precision not available");
  return HBPC_OK;
}

void fill_params(hbpc_ctx* x) {
  DGParams<double>& p = x->prm;
  std::memset(&p, 0, sizeof(p));
  const int P = x->P;
  for (int m = 0; m < 3; ++m) p.n[m] = m < x->dim ? x->mesh.n[m] : 1;
  p.nE = int(x->nE);
  for (int m = 0; m < x->dim; ++m) {
    const double h = (x->mesh.hi[m] - x->mesh.lo[m]) / x->mesh.n[m];
    const double sc = -2.0 / h;
    const double av = x->phys.law == HBPC_LAW_ADVECTION ? x->phys.a[m] : 1.0;
    for (int i = 0; i < P; ++i) {
      for (int l = 0; l < P; ++l) p.Dvol[m][i][l] = sc * av * x->basis.Dhat[i * P + l];
      p.sp[m][i] = sc * x->basis.lp[i] / x->basis.w[i];
      p.sm[m][i] = sc * x->basis.lm[i] / x->basis.w[i];
    }
    for (int v = 0; v < 5; ++v) {
      double lam = 1.0;
      if (x->phys.law == HBPC_LAW_ADVECTION) lam = std::fabs(x->phys.a[m]);
      else if (x->phys.law == HBPC_LAW_EULER) lam = (v == 0 || v == x->nv - 1) ? 1.0 / x->phys.eps : 1.0;
      p.lam[m][v] = x->phys.lf_scale * lam;
    }
    p.a[m] = x->phys.a[m];
  }
  for (int i = 0; i < P; ++i) { p.lp[i] = x->basis.lp[i]; p.lm[i] = x->basis.lm[i]; }
  p.gamma = x->phys.gamma;
  p.gm1 = x->phys.gamma - 1.0;
  p.eps2 = x->phys.eps * x->phys.eps;
  p.inv_eps2 = 1.0 / p.eps2;
  p.inv_eps = 1.0 / x->phys.eps;
  p.rusanov = x->phys.flux == HBPC_FLUX_RUSANOV ? 1 : 0;
}


// ---------------------------------------------------------------------------
// Allocation-free Jacobian-vector product.  Its scratch (R1(W) and R2(W, S) at
// the linearisation point, the per-block partial sums of the ||dW||, ||dS||
// reduction, the reduction ticket and a few scalars) lives in one file-scope
// device array instead of memory obtained from cudaMalloc.
// ---------------------------------------------------------------------------
constexpr long long kNoAllocMaxDof = 1LL << 18;   // n_dof limit (262,144 values)
constexpr int kNoAllocMaxBlocks = 512;            // reduction blocks
constexpr size_t kNoAllocR1 = 0;                                          // doubles
constexpr size_t kNoAllocR2 = kNoAllocR1 + size_t(kNoAllocMaxDof);
constexpr size_t kNoAllocPartial = kNoAllocR2 + size_t(kNoAllocMaxDof);   // blocks x 4
constexpr size_t kNoAllocC12 = kNoAllocPartial + size_t(kNoAllocMaxBlocks) * 4;
constexpr size_t kNoAllocNrm = kNoAllocC12 + 4;
constexpr size_t kNoAllocState = kNoAllocNrm + 4;                         // GmresState
constexpr size_t kNoAllocTicket = kNoAllocState + (sizeof(GmresState) + 7) / 8;
constexpr size_t kNoAllocBytes = (kNoAllocTicket + 1) * sizeof(double);  // about 4.2 MB

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device.  The first call
// on a device resolves it (cudaGetSymbolAddress, with that device current);
// later calls reuse the cached address.
hbpc_status noalloc_scratch(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return fail(nullptr, HBPC_ERR_UNSUPPORTED, "device index beyond the allocation-free table");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(nullptr, e, "cudaGetSymbolAddress(scratch)");
    g_noalloc_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_noalloc_addr[dev]);
  return HBPC_OK;
}

}  // namespace

extern "C" {

hbpc_status hbpc_basis(int N, int nodes, double* xi, double* w, double* Dhat, double* lm, double* lp) {
  Basis1D b;
  if (nodes != HBPC_NODES_LOBATTO && nodes != HBPC_NODES_GAUSS)
    return fail(nullptr, HBPC_ERR_INVALID_ARG, "unknown node family");
  if (!basis_1d(N, nodes, b)) return fail(nullptr, HBPC_ERR_INVALID_ARG, "N must satisfy 1 <= N <= 7");
  const int p = N + 1;
  if (xi) std::memcpy(xi, b.xi.data(), p * sizeof(double));
  if (w) std::memcpy(w, b.w.data(), p * sizeof(double));
  if (Dhat) std::memcpy(Dhat, b.Dhat.data(), p * p * sizeof(double));
  if (lm) std::memcpy(lm, b.lm.data(), p * sizeof(double));
  if (lp) std::memcpy(lp, b.lp.data(), p * sizeof(double));
  return HBPC_OK;
}

hbpc_status hbpc_create(hbpc_ctx** out, const hbpc_mesh* mesh, int N, int nodes,
                        const hbpc_physics* phys, const hbpc_solver* solver, void* cuda_stream) {
  if (!out) return fail(nullptr, HBPC_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  hbpc_status s = validate(mesh, N, nodes, phys, solver);
  if (s != HBPC_OK) return s;
  hbpc_ctx* x = new (std::nothrow) hbpc_ctx();
  if (!x) return fail(nullptr, HBPC_ERR_OOM, "host allocation failed");
  x->mesh = *mesh; x->phys = *phys; x->sol = *solver;
  x->N = N; x->P = N + 1; x->nodes = nodes; x->dim = mesh->dim;
  x->nv = phys->law == HBPC_LAW_EULER ? mesh->dim + 2 : 1;
  x->nE = 1;
  for (int m = 0; m < x->dim; ++m) x->nE *= mesh->n[m];
  long long nn = 1;
  for (int m = 0; m < x->dim; ++m) nn *= x->P;
  x->ndof = x->nE * x->nv * nn;
  x->stream = static_cast<cudaStream_t>(cuda_stream);
  if (const char* v = std::getenv("HBPC_VERBOSE")) x->verbose = std::atoi(v);
  if (!basis_1d(N, nodes, x->basis)) { delete x; return fail(nullptr, HBPC_ERR_INVALID_ARG, "basis"); }
  if (!get_ops(phys->law, x->dim, x->P, nodes == HBPC_NODES_LOBATTO, x->ops)) {
    delete x;
    return fail(nullptr, HBPC_ERR_UNSUPPORTED, "this (law, dim, N, node family) is not compiled in");
  }
  if (x->nE > (1LL << 30)) { delete x; return fail(nullptr, HBPC_ERR_INVALID_ARG, "mesh too large"); }
  tableau(solver->q, x);
  fill_params(x);
  const size_t n = size_t(x->ndof), n2 = 2 * n;
  const int m = solver->gmres_restart;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  x->nblocks = std::max(1, std::min<int>(2 * sms, int((n2 + 1023) / 1024)));
  x->nb = int(x->ndof / x->nE);
  if (solver->pc == HBPC_PC_BJEXT) {
    const int epb = std::max(1, 256 / x->nb);
    x->pc_threads = ((epb * x->nb + 31) / 32) * 32;
    x->pc_grid = int((x->nE + epb - 1) / epb);
    x->pc_smem = size_t(epb) * 4 * x->nb * sizeof(double);
  }
  const int prows = std::max(x->nblocks, x->pc_grid);
  hbpc_status e = HBPC_OK;
  if ((e = dmalloc(x, &x->Wn, n)) || (e = dmalloc(x, &x->X, n2)) || (e = dmalloc(x, &x->G, n2)) ||
      (e = dmalloc(x, &x->r1, n)) || (e = dmalloc(x, &x->r2, n)) || (e = dmalloc(x, &x->dX, n2)) ||
      (e = dmalloc(x, &x->bvec, n)) || (e = dmalloc(x, &x->stage, size_t(2) * x->s * 3 * n)) ||
      (e = dmalloc(x, &x->V, size_t(m + 1) * n2))) {
    g_create_error = x->err;
    free_all(x); delete x; return e;
  }
  const size_t nsmall = size_t(m + 1) * m + 3 * m + 8 * (m + 3) + 24;
  if (solver->pc == HBPC_PC_BJEXT) {
    const size_t blk = size_t(x->nE) * x->nb * x->nb;
    if ((e = dmalloc(x, &x->Jpc, blk)) || (e = dmalloc(x, &x->Mpc, blk)) || (e = dmalloc(x, &x->Z, n2)) ||
        (e = dmalloc(x, &x->singular, 1))) {
      g_create_error = x->err;
      free_all(x); delete x; return e;
    }
    const size_t nbz = size_t(x->nb);
    cudaFuncSetAttribute(k_pc_form_S, cudaFuncAttributeMaxDynamicSharedMemorySize, int(nbz * nbz * sizeof(double)));
    cudaFuncSetAttribute(k_pc_invert, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         int((nbz * nbz + nbz) * sizeof(double) + nbz * sizeof(int)));
  }
  if ((e = dmalloc(x, &x->small, nsmall)) || (e = dmalloc(x, &x->partial, size_t(prows) * (m + 3))) ||
      (e = dmalloc(x, &x->ticket, 1)) || (e = dmalloc(x, &x->st, 1))) {
    g_create_error = x->err;
    free_all(x); delete x; return e;
  }
  if (cudaMallocHost(reinterpret_cast<void**>(&x->st_host), sizeof(GmresState)) != cudaSuccess) {
    g_create_error = "cudaMallocHost failed";
    free_all(x); delete x; return HBPC_ERR_OOM;
  }
  double* q = x->small;
  Krylov& K = x->K;
  K.V = x->V; K.ld = n2; K.n2 = n2; K.half = n; K.m = m;
  K.H = q; q += size_t(m + 1) * m;
  K.cs = q; q += m;
  K.sn = q; q += m;
  K.y = q; q += m;
  K.g = q; q += m + 3;
  K.vscale = q; q += m + 3;
  K.nrmW = q; q += m + 3;
  K.nrmS = q; q += m + 3;
  K.hc = q; q += m + 3;
  x->c12 = q; q += 4;
  x->dxn = q; q += 4;
  x->zn = q; q += 4;
  K.st = x->st; K.partial = x->partial; K.ticket = x->ticket; K.nblocks = x->nblocks;
  cudaError_t ce = cudaMemsetAsync(x->small, 0, nsmall * sizeof(double), x->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(x->ticket, 0, sizeof(unsigned), x->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(x->st, 0, sizeof(GmresState), x->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(x->Wn, 0, n * sizeof(double), x->stream);
  if (ce == cudaSuccess && x->singular) ce = cudaMemsetAsync(x->singular, 0, sizeof(int), x->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(x->stream);
  if (ce != cudaSuccess) {
    g_create_error = std::string("initialisation: ") + cudaGetErrorString(ce);
    free_all(x); delete x; return HBPC_ERR_CUDA;
  }
  *out = x;
  return HBPC_OK;
}

void hbpc_destroy(hbpc_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  free_all(ctx);
  delete ctx;
}

long long hbpc_ndof(const hbpc_ctx* ctx) { return ctx ? ctx->ndof : 0; }
int hbpc_nvar(const hbpc_ctx* ctx) { return ctx ? ctx->nv : 0; }

hbpc_status hbpc_node_coords(const hbpc_ctx* ctx, double* xo) {
  if (!ctx || !xo) return HBPC_ERR_INVALID_ARG;
  const int d = ctx->dim, P = ctx->P;
  long long nn = 1;
  for (int m = 0; m < d; ++m) nn *= P;
  const long long per = ctx->nE * nn;
  for (long long e = 0; e < ctx->nE; ++e) {
    long long ec[3] = {0, 0, 0};
    ec[0] = e % ctx->mesh.n[0];
    if (d > 1) ec[1] = (e / ctx->mesh.n[0]) % ctx->mesh.n[1];
    if (d > 2) ec[2] = e / (ctx->mesh.n[0] * (long long)ctx->mesh.n[1]);
    for (long long node = 0; node < nn; ++node) {
      long long id[3] = {node % P, (node / P) % P, node / (P * P)};
      for (int m = 0; m < d; ++m) {
        const double h = (ctx->mesh.hi[m] - ctx->mesh.lo[m]) / ctx->mesh.n[m];
        xo[m * per + e * nn + node] = ctx->mesh.lo[m] + h * ec[m] + 0.5 * h * (ctx->basis.xi[id[m]] + 1.0);
      }
    }
  }
  return HBPC_OK;
}

hbpc_status hbpc_set_state(hbpc_ctx* ctx, const double* w, int on_device) {
  if (!ctx || !w) return HBPC_ERR_INVALID_ARG;
  HBPC_CK(ctx, cudaMemcpyAsync(ctx->Wn, w, size_t(ctx->ndof) * sizeof(double),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
  return sync(ctx, "set_state");
}

hbpc_status hbpc_get_state(const hbpc_ctx* cctx, double* w, int on_device) {
  hbpc_ctx* ctx = const_cast<hbpc_ctx*>(cctx);
  if (!ctx || !w) return HBPC_ERR_INVALID_ARG;
  HBPC_CK(ctx, cudaMemcpyAsync(w, ctx->Wn, size_t(ctx->ndof) * sizeof(double),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
  return sync(ctx, "get_state");
}

hbpc_status hbpc_set_time(hbpc_ctx* ctx, double t) {
  if (!ctx) return HBPC_ERR_INVALID_ARG;
  ctx->stats.t = t;
  return HBPC_OK;
}

hbpc_status hbpc_step(hbpc_ctx* ctx, int n_steps) {
  if (!ctx || n_steps < 0) return HBPC_ERR_INVALID_ARG;
  for (int i = 0; i < n_steps; ++i) {
    hbpc_status s = hbpc_one_step(ctx);
    if (s != HBPC_OK) return s;
    ctx->stats.steps += 1;
    ctx->stats.t += ctx->sol.dt;
  }
  return HBPC_OK;
}

hbpc_status hbpc_eval_R1(hbpc_ctx* ctx, const double* w, double* r) {
  if (!ctx || !w || !r) return HBPC_ERR_INVALID_ARG;
  ctx->ops.r1(ctx->prm, w, r, ctx->stream);
  HBPC_LAUNCH_CK(ctx, "eval_R1");
  ctx->stats.r1_evals += 1;
  return sync(ctx, "eval_R1");
}

hbpc_status hbpc_eval_R2(hbpc_ctx* ctx, const double* w, const double* s, double* r) {
  if (!ctx || !w || !s || !r) return HBPC_ERR_INVALID_ARG;
  ctx->ops.r2(ctx->prm, w, s, r, ctx->stream);
  HBPC_LAUNCH_CK(ctx, "eval_R2");
  ctx->stats.r2_evals += 1;
  return sync(ctx, "eval_R2");
}

hbpc_status hbpc_eval_G(hbpc_ctx* ctx, const double* b, double alpha1, double alpha2,
                        const double* X, double* G) {
  if (!ctx || !b || !X || !G) return HBPC_ERR_INVALID_ARG;
  const long long n = ctx->ndof;
  const double dt = ctx->sol.dt;
  HBPC_CK(ctx, cudaMemcpyAsync(ctx->X, X, size_t(2 * n) * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  hbpc_status s = residual(ctx, b, alpha1 * dt, alpha2 * dt * dt / 2.0);
  if (s != HBPC_OK) return s;
  HBPC_CK(ctx, cudaMemcpyAsync(G, ctx->G, size_t(2 * n) * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  return sync(ctx, "eval_G");
}

hbpc_status hbpc_eval_Jv(hbpc_ctx* ctx, double alpha1, double alpha2, const double* X,
                         const double* dX, double* out) {
  if (!ctx || !X || !dX || !out) return HBPC_ERR_INVALID_ARG;
  const long long n = ctx->ndof;
  const size_t n2 = size_t(2 * n);
  const double dt = ctx->sol.dt;
  const double c1 = alpha1 * dt, c2 = alpha2 * dt * dt / 2.0;
  HBPC_RUN(ctx, HBPC_PHASE_VECTOR, 1, k_set2<<<1, 32, 0, ctx->stream>>>(ctx->c12, c1, c2));
  HBPC_CK(ctx, cudaMemcpyAsync(ctx->X, X, n2 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  // R1(W), R2(W, S) at X (b does not enter Jv; use X's own W as a dummy)
  ctx->ops.residual(ctx->prm, ctx->X, ctx->X + n, ctx->X, c1, c2, ctx->G, ctx->G + n, ctx->r1, ctx->r2,
                    ctx->stream);
  HBPC_LAUNCH_CK(ctx, "Jv residual");
  HBPC_CK(ctx, cudaMemcpyAsync(ctx->dX, dX, n2 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  hbpc_status s = norms(ctx, ctx->dX, n2, ctx->dxn);
  if (s != HBPC_OK) return s;
  JvInput z{};
  z.V = ctx->dX; z.ld = n2; z.half = size_t(n);
  z.nrmW = ctx->dxn + 1; z.nrmS = ctx->dxn + 2;
  z.out = out; z.out_ld = n2; z.out_offset = 0;
  if ((s = apply_jv(ctx, z)) != HBPC_OK) return s;
  return sync(ctx, "eval_Jv");
}

hbpc_status hbpc_eval_pc(hbpc_ctx* ctx, double alpha1, double alpha2, const double* X,
                         const double* in, double* out) {
  if (!ctx || !X || !in || !out) return HBPC_ERR_INVALID_ARG;
  if (ctx->sol.pc != HBPC_PC_BJEXT) return fail(ctx, HBPC_ERR_INVALID_ARG, "context has no preconditioner");
  const long long n = ctx->ndof;
  const size_t n2 = size_t(2 * n);
  const double dt = ctx->sol.dt;
  const double c1 = alpha1 * dt, c2 = alpha2 * dt * dt / 2.0;
  HBPC_RUN(ctx, HBPC_PHASE_VECTOR, 1, k_set2<<<1, 32, 0, ctx->stream>>>(ctx->c12, c1, c2));
  HBPC_CK(ctx, cudaMemcpyAsync(ctx->X, X, n2 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  ctx->pc_built = false;
  hbpc_status s = pc_build(ctx, ctx->X, c1, c2);
  if (s != HBPC_OK) return s;
  HBPC_CK(ctx, cudaMemcpyAsync(ctx->Z, in, n2 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  if ((s = pc_apply(ctx, ctx->Z, nullptr, nullptr, out, 0, nullptr)) != HBPC_OK) return s;
  return sync(ctx, "eval_pc");
}

hbpc_status hbpc_newton_solve(hbpc_ctx* ctx, const double* b, double alpha1, double alpha2,
                              const double* W0, double* W_out, double* S_out) {
  if (!ctx || !b || !W0 || !W_out) return HBPC_ERR_INVALID_ARG;
  const long long n = ctx->ndof;
  HBPC_CK(ctx, cudaMemcpyAsync(ctx->bvec, b, size_t(n) * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  hbpc_status s = newton(ctx, ctx->bvec, alpha1, alpha2, W0);
  if (s != HBPC_OK) return s;
  HBPC_CK(ctx, cudaMemcpyAsync(W_out, ctx->X, size_t(n) * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  if (S_out)
    HBPC_CK(ctx, cudaMemcpyAsync(S_out, ctx->X + n, size_t(n) * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  return sync(ctx, "newton_solve");
}

hbpc_status hbpc_get_stats(const hbpc_ctx* ctx, hbpc_stats* out) {
  if (!ctx || !out) return HBPC_ERR_INVALID_ARG;
  *out = ctx->stats;
  return HBPC_OK;
}

hbpc_status hbpc_reset_stats(hbpc_ctx* ctx) {
  if (!ctx) return HBPC_ERR_INVALID_ARG;
  const double t = ctx->stats.t;
  ctx->stats = hbpc_stats{};
  ctx->stats.t = t;
  return HBPC_OK;
}

hbpc_status hbpc_profile_enable(hbpc_ctx* ctx, int enable) {
  if (!ctx) return HBPC_ERR_INVALID_ARG;
  hbpc_status s = sync(ctx, "profile_enable");
  if (s != HBPC_OK) return s;
  ctx->prof.on = enable != 0;
  for (int i = 0; i < HBPC_NPHASES; ++i) { ctx->prof.ms[i] = 0.0; ctx->prof.cnt[i] = 0; }
  return HBPC_OK;
}

hbpc_status hbpc_profile_get(hbpc_ctx* ctx, double* ms, long long* launches, int n_phases) {
  if (!ctx || n_phases < 0) return HBPC_ERR_INVALID_ARG;
  hbpc_status s = sync(ctx, "profile_get");
  if (s != HBPC_OK) return s;
  for (int i = 0; i < n_phases && i < HBPC_NPHASES; ++i) {
    if (ms) ms[i] = ctx->prof.ms[i];
    if (launches) launches[i] = ctx->prof.cnt[i];
  }
  return HBPC_OK;
}

hbpc_status hbpc_eval_Jv_noalloc(const hbpc_mesh* mesh, int N, int nodes, const hbpc_physics* phys,
                                 double dt, double alpha1, double alpha2, const double* X,
                                 const double* dX, double* out, void* cuda_stream) {
  if (!X || !dX || !out) return fail(nullptr, HBPC_ERR_INVALID_ARG, "null pointer");
  hbpc_solver so{};
  so.q = 4; so.kmax = 0; so.dt = dt;
  so.tol_newton_rel = 1e-12; so.tol_newton_abs = 0.0; so.tol_gmres_rel = 1e-5;
  so.gmres_restart = 1; so.gmres_max_iter = 1; so.newton_max_iter = 1;
  so.pc = HBPC_PC_NONE; so.precision = HBPC_PREC_FP64;
  hbpc_status st = validate(mesh, N, nodes, phys, &so);
  if (st != HBPC_OK) return st;
  // host-side description of the discretisation (no device memory)
  hbpc_ctx x;
  x.mesh = *mesh; x.phys = *phys; x.sol = so;
  x.N = N; x.P = N + 1; x.nodes = nodes; x.dim = mesh->dim;
  x.nv = phys->law == HBPC_LAW_EULER ? mesh->dim + 2 : 1;
  x.nE = 1;
  for (int m = 0; m < x.dim; ++m) x.nE *= mesh->n[m];
  long long nn = 1;
  for (int m = 0; m < x.dim; ++m) nn *= x.P;
  x.ndof = x.nE * x.nv * nn;
  if (x.ndof > kNoAllocMaxDof)
    return fail(nullptr, HBPC_ERR_INVALID_ARG,
                "n_dof exceeds the allocation-free limit of 262144 values; use hbpc_eval_Jv");
  if (!basis_1d(N, nodes, x.basis)) return fail(nullptr, HBPC_ERR_INVALID_ARG, "basis");
  if (!get_ops(phys->law, x.dim, x.P, nodes == HBPC_NODES_LOBATTO, x.ops))
    return fail(nullptr, HBPC_ERR_UNSUPPORTED, "this (law, dim, N, node family) is not compiled in");
  fill_params(&x);
  unsigned char* base = nullptr;
  if ((st = noalloc_scratch(&base)) != HBPC_OK) return st;
  double* scr = reinterpret_cast<double*>(base);
  const cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  const long long n = x.ndof;
  const size_t n2 = size_t(2 * n);
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  Krylov K{};
  K.m = 1;   // partial stride m + 3 = 4
  K.partial = scr + kNoAllocPartial;
  K.st = reinterpret_cast<GmresState*>(scr + kNoAllocState);
  K.ticket = reinterpret_cast<unsigned*>(scr + kNoAllocTicket);
  K.nblocks = std::max(1, std::min<int>({2 * sms, int((n2 + 1023) / 1024), kNoAllocMaxBlocks}));
  double* c12 = scr + kNoAllocC12;
  double* nrm = scr + kNoAllocNrm;
  const double c1 = alpha1 * dt, c2 = alpha2 * dt * dt / 2.0;
  auto ck = [&](cudaError_t e, const char* what) -> hbpc_status {
    return e == cudaSuccess ? HBPC_OK : cuda_fail(nullptr, e, what);
  };
  // the shared array keeps the previous call's contents: the ticket must start at 0
  if ((st = ck(cudaMemsetAsync(K.ticket, 0, sizeof(unsigned), stream), "clear ticket")) != HBPC_OK) return st;
  k_set2<<<1, 32, 0, stream>>>(c12, c1, c2);
  // R1(W), R2(W, S) at X into the scratch (G goes to `out`, overwritten below)
  x.ops.residual(x.prm, X, X + n, X, c1, c2, out, out + n, scr + kNoAllocR1, scr + kNoAllocR2, stream);
  k_norms<<<K.nblocks, kVecThreads, 0, stream>>>(dX, n2, size_t(n), K, nullptr);
  k_sqrt_norms<<<1, 32, 0, stream>>>(K.st, nrm);
  if ((st = ck(cudaGetLastError(), "noalloc launches")) != HBPC_OK) return st;
  JvInput z{};
  z.V = dX; z.ld = n2; z.half = size_t(n);
  z.nrmW = nrm + 1; z.nrmS = nrm + 2;
  z.out = out; z.out_ld = n2; z.out_offset = 0;
  JvCoef cf;
  cf.c1 = c12; cf.c2 = c12 + 1;
  cf.sqrt_eps_machine = std::sqrt(std::ldexp(1.0, -52));
  cf.eps_ref = phys->eps;
  if (x.ops.jv_linear) x.ops.jv_linear(x.prm, z, cf, stream);
  else x.ops.jv_fd(x.prm, X, X + n, scr + kNoAllocR1, scr + kNoAllocR2, z, cf, stream);
  if ((st = ck(cudaGetLastError(), "noalloc jv")) != HBPC_OK) return st;
  return ck(cudaStreamSynchronize(stream), "noalloc sync");
}

const char* hbpc_last_error(const hbpc_ctx* ctx) {
  if (!ctx) return g_create_error.c_str();
  return ctx->err.c_str();
}

}  // extern "C"
