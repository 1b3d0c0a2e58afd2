// Device-driven HBPC step: the control kernels of the one-graph form of a
// time step (Algorithm 1 with the Newton iteration of Eq. 17 and restarted
// GMRES as conditional WHILE/IF graph nodes).  Every decision the host loop
// takes after reading the GMRES state or the Newton norms is taken here by a
// single thread, which sets the conditional handle of the loop or branch that
// follows; the step's outcome (error, iteration counts, kernels run) collects
// in a StepCtl block that the host reads once, after the graph.
// Included by exactly one translation unit.
#pragma once
#include <cuda_runtime.h>

#include "krylov_common.cuh"

namespace hbpc {

struct StepCtl {
  int err;              // 0, or the hbpc_status code that ended the step
  int where;            // 1 initial Newton residual, 2 Newton residual, 3 GMRES residual, 4 Newton cap
  int newton_it;        // Newton iterations of the solve in progress
  int jprev;            // Arnoldi columns of the current GMRES cycle already counted
  double g0;            // single problem: ||G(X^0)||
  double dw;            // single problem: ||dW|| of the last update
  long long newton_solves, newton_its, gmres_its, arnoldi_cols, launches;
};

constexpr int kSgErrNonfinite = 5;       // HBPC_ERR_NONFINITE
constexpr int kSgErrNoConvergence = 4;   // HBPC_ERR_NO_CONVERGENCE

__device__ __forceinline__ bool sg_finite(double v) { return v == v && v - v == 0.0; }
__device__ __forceinline__ long long sg_cols(int j0, int j1) {
  return j1 <= j0 ? 0 : (long long)(j1 - j0) * (j0 + j1 + 1) / 2;
}

__global__ void k_sg_reset(StepCtl* c) {
  if (threadIdx.x == 0) {
    c->err = 0; c->where = 0; c->newton_it = 0; c->jprev = 0; c->g0 = 0.0; c->dw = 0.0;
    c->newton_solves = 0; c->newton_its = 0; c->gmres_its = 0; c->arnoldi_cols = 0; c->launches = 1;
  }
}

// Kernels of a loop body the control kernels do not see (a restart branch).
__global__ void k_sg_count(StepCtl* c, int n) {
  if (threadIdx.x == 0) c->launches += n;
}

// dst = src (n doubles) unless the step failed: the state of the step only
// replaces w^{n-1} when every solve succeeded.
__global__ void k_sg_copy_if_ok(const double* __restrict__ src, double* __restrict__ dst, size_t n,
                                const StepCtl* c) {
  if (c->err) return;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    dst[i] = src[i];
}

// ---- Newton (single problem: the norms in st->nrm) ------------------------
__global__ void k_sg_newton_begin(const GmresState* st, StepCtl* c, cudaGraphConditionalHandle h, int n) {
  if (threadIdx.x != 0) return;
  c->launches += n;
  const double g0 = sqrt(st->nrm[0]);
  c->g0 = g0;
  c->newton_it = 0;
  if (!sg_finite(g0) && !c->err) { c->err = kSgErrNonfinite; c->where = 1; }
  if (!c->err) c->newton_solves += 1;
  cudaGraphSetConditional(h, (!c->err && g0 > 0.0) ? 1u : 0u);
}

__global__ void k_sg_save_dw(const GmresState* st, StepCtl* c) {
  if (threadIdx.x == 0) c->dw = sqrt(st->nrm[1]);
}

// After an update and the new residual: the stopping tests of Sec. 3.2.1
// (||G|| <= tol_rel ||G^0|| or ||dW|| <= tol_abs) and the iteration cap.
__global__ void k_sg_newton_check(const GmresState* st, StepCtl* c, cudaGraphConditionalHandle h, double tol_rel,
                                  double tol_abs, int max_it, int n) {
  if (threadIdx.x != 0) return;
  c->launches += n;
  c->newton_it += 1;
  c->newton_its += 1;
  const double gn = sqrt(st->nrm[0]);
  bool cont = true;
  if (!sg_finite(gn) || !sg_finite(c->dw)) {
    if (!c->err) { c->err = kSgErrNonfinite; c->where = 2; }
    cont = false;
  } else if (gn <= tol_rel * c->g0 || c->dw <= tol_abs) {
    cont = false;
  }
  if (c->err) cont = false;
  if (cont && c->newton_it >= max_it) {
    c->err = kSgErrNoConvergence; c->where = 4;
    cont = false;
  }
  cudaGraphSetConditional(h, cont ? 1u : 0u);
}

// ---- Newton (batch group: per-instance norms in inrm = (||G_i||^2, ||dW_i||^2)) ----
// Active instances and the right-hand side scaling of the next GMRES: 1 for
// per-instance GMRES, 1 / ||G_i|| for the shared one, 0 for a frozen instance.
__global__ void __launch_bounds__(256) k_sg_newton_begin_batch(int ni, const double* __restrict__ inrm,
                                                               double* __restrict__ g0, int* __restrict__ active,
                                                               double* __restrict__ iscale, int per_instance,
                                                               StepCtl* c, cudaGraphConditionalHandle h, int n) {
  __shared__ int s_act, s_bad;
  if (threadIdx.x == 0) { s_act = 0; s_bad = 0; }
  __syncthreads();
  for (int i = threadIdx.x; i < ni; i += blockDim.x) {
    const double g = sqrt(inrm[2 * i]);
    if (!sg_finite(g)) atomicExch(&s_bad, 1);
    g0[i] = g;
    active[i] = g > 0.0 ? 1 : 0;
    iscale[i] = !(g > 0.0) ? 0.0 : per_instance ? 1.0 : 1.0 / g;
    if (g > 0.0) atomicAdd(&s_act, 1);
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  c->launches += n;
  c->newton_it = 0;
  if (s_bad && !c->err) { c->err = kSgErrNonfinite; c->where = 1; }
  if (!c->err) c->newton_solves += 1;
  cudaGraphSetConditional(h, (!c->err && s_act > 0) ? 1u : 0u);
}

__global__ void k_sg_save_dw_batch(int ni, const double* __restrict__ inrm, double* __restrict__ dw) {
  for (int i = threadIdx.x; i < ni; i += blockDim.x) dw[i] = sqrt(inrm[2 * i + 1]);
}

__global__ void __launch_bounds__(256) k_sg_newton_check_batch(int ni, const double* __restrict__ inrm,
                                                               const double* __restrict__ dw,
                                                               const double* __restrict__ g0,
                                                               int* __restrict__ active, double* __restrict__ iscale,
                                                               int per_instance, StepCtl* c,
                                                               cudaGraphConditionalHandle h, double tol_rel,
                                                               double tol_abs, int max_it, int n) {
  __shared__ int s_act, s_bad;
  if (threadIdx.x == 0) { s_act = 0; s_bad = 0; }
  __syncthreads();
  for (int i = threadIdx.x; i < ni; i += blockDim.x) {
    if (!active[i]) { iscale[i] = 0.0; continue; }
    const double gn = sqrt(inrm[2 * i]);
    if (!sg_finite(gn) || !sg_finite(dw[i])) {
      atomicExch(&s_bad, 1);
      continue;
    }
    if (gn <= tol_rel * g0[i] || dw[i] <= tol_abs) {
      active[i] = 0;
      iscale[i] = 0.0;
    } else {
      iscale[i] = per_instance ? 1.0 : 1.0 / gn;
      atomicAdd(&s_act, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  c->launches += n;
  c->newton_it += 1;
  c->newton_its += 1;
  if (s_bad && !c->err) { c->err = kSgErrNonfinite; c->where = 2; }
  bool cont = !c->err && s_act > 0;
  if (cont && c->newton_it >= max_it) {
    c->err = kSgErrNoConvergence; c->where = 4;
    cont = false;
  }
  cudaGraphSetConditional(h, cont ? 1u : 0u);
}

// ---- restarted GMRES ---------------------------------------------------------
__global__ void k_sg_gmres_begin(StepCtl* c, cudaGraphConditionalHandle h, int n) {
  if (threadIdx.x != 0) return;
  c->launches += n;
  c->jprev = 0;
  cudaGraphSetConditional(h, c->err ? 0u : 1u);
}

// After a batch of columns: count them, stop on a non-finite residual
// (unless the residual is per instance), open the cycle-end branch once the
// cycle is done.
__global__ void k_sg_gmres_tick(const GmresState* st, StepCtl* c, cudaGraphConditionalHandle h_loop,
                                cudaGraphConditionalHandle h_end, int check_resid, int n) {
  if (threadIdx.x != 0) return;
  c->launches += n;
  c->arnoldi_cols += sg_cols(c->jprev, st->j);
  c->jprev = st->j;
  if (check_resid && !sg_finite(st->resid) && !c->err) { c->err = kSgErrNonfinite; c->where = 3; }
  cudaGraphSetConditional(h_end, (!c->err && st->done) ? 1u : 0u);
  cudaGraphSetConditional(h_loop, c->err ? 0u : 1u);
}

// End of a cycle: the solve ends when converged or at its iteration cap
// (Newton goes on either way), otherwise the restart branch runs.
__global__ void k_sg_gmres_end(const GmresState* st, StepCtl* c, cudaGraphConditionalHandle h_loop,
                               cudaGraphConditionalHandle h_restart, int n) {
  if (threadIdx.x != 0) return;
  c->launches += n;
  const bool finish = st->converged || st->its >= st->max_its;
  if (finish) c->gmres_its += st->its;
  c->jprev = 0;
  cudaGraphSetConditional(h_loop, finish ? 0u : 1u);
  cudaGraphSetConditional(h_restart, finish ? 0u : 1u);
}

}  // namespace hbpc
