// C-ABI of libhbpc (include/hbpc.h): context set-up, the Newton-GMRES stage
// solve (Sec. 3.2, 4.2) and the HBPC(q, k_max) driver (Algorithm 1, Sec. 2.1).
// The host only sequences launches; every vector of the method lives on the
// device and the per-iteration GMRES state is device-resident, so the host
// waits on the GPU once per batch of GMRES iterations and once per Newton
// iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdint>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <random>
#include <string>
#include <thread>
#include <vector>

#include "../../include/hbpc.h"
#include "dg_ops.cuh"
#include "hbpc_internal.h"
#include "krylov.cuh"
#include "batch_krylov.cuh"
#include "bjext_kernels.cuh"
#include "bjext_tc.cuh"
#include "step_graph.cuh"
#include "mlp.cuh"

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

// Schur form (Sec. 3.2.4) helpers on 2 n vectors whose second half is the
// sigma part.  A step is skipped when *skip != 0 (the GMRES cycle is done).
// out = scale[j] * V[j] (j = *jidx), the column of the Krylov basis
__global__ void k_gather_col(const double* V, const int* jidx, const double* scale, double* out, size_t n2,
                             const int* skip) {
  if (skip && *skip) return;
  const int j = *jidx;
  const double sc = scale[j];
  const double* v = V + size_t(j) * n2;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n2; i += size_t(gridDim.x) * blockDim.x)
    out[i] = sc * v[i];
}
// zero the sigma half of column (*jidx + off) of V (jidx null: of V itself)
__global__ void k_zero_half(double* V, const int* jidx, int off, size_t n, const int* skip) {
  if (skip && *skip) return;
  double* v = V + (jidx ? size_t(*jidx + off) * 2 * n : 0) + n;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    v[i] = 0.0;
}
// y_S = -o_S (o = the extended product on (z, 0), whose sigma half is -J z):
// y = (z, J z) in place of y = (z, 0)
__global__ void k_schur_pair(double* y, const double* o, size_t n, const int* skip) {
  if (skip && *skip) return;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    y[n + i] = -o[n + i];
}
// out = (-G1 - c2 o_S, 0) with o_S = -J G2: the Schur right-hand side
// -G1 + c2 (dR2/dsigma) G2 (R2 is linear in sigma, and dR2/dsigma = dR1/dW)
__global__ void k_schur_rhs(const double* G, const double* o, const double* c12, double* out, size_t n) {
  const double c2 = c12[1];
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    out[i] = -G[i] - c2 * o[n + i];
    out[n + i] = 0.0;
  }
}
// dX_S = -G2 - o_S (o_S = -J dW): the sigma increment -G2 + (dR1/dW) dW
__global__ void k_schur_sigma(const double* G, const double* o, double* dX, size_t n) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    dX[n + i] = -G[n + i] - o[n + i];
}
// y_W += x_W (first halves only)
__global__ void k_add_half(const double* x, double* y, size_t n) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    y[i] += x[i];
}
// out = (r_W - p_W, 0): the restart residual of the Schur system
__global__ void k_schur_restart(const double* r, const double* p, double* out, size_t n) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    out[i] = r[i] - p[i];
    out[n + i] = 0.0;
  }
}

__global__ void k_set2(double* p, double a, double b) {
  if (threadIdx.x == 0) { p[0] = a; p[1] = b; }
}

// sqrt of the three squared norms in st->nrm into out[0..2]
__global__ void k_sqrt_norms(const GmresState* st, double* out) {
  if (threadIdx.x < 3) out[threadIdx.x] = sqrt(st->nrm[threadIdx.x]);
}

// Batches: per-instance squared norms of a 2 n_dof vector v = (vW, vS), one
// block per instance (fixed-order reduction): out[2 i] = |v_i|^2 over both
// halves, out[2 i + 1] = |vW_i|^2.  range[2 i], range[2 i + 1]: first value and
// count of instance i in a half.
constexpr int kInstThreads = 512;
__global__ void __launch_bounds__(kInstThreads) k_inst_sqnorms(const double* __restrict__ v, size_t half,
                                                             const long long* __restrict__ range,
                                                             double* __restrict__ out) {
  const int i = blockIdx.x;
  const long long a = range[2 * i], cnt = range[2 * i + 1];
  double sw = 0.0, ss = 0.0;
  for (long long t = threadIdx.x; t < cnt; t += blockDim.x) {
    const double x = v[a + t], y = v[half + a + t];
    sw += x * x;
    ss += y * y;
  }
  __shared__ double rw[kInstThreads / 32], rs[kInstThreads / 32];
  sw = warp_sum(sw);
  ss = warp_sum(ss);
  if ((threadIdx.x & 31) == 0) { rw[threadIdx.x >> 5] = sw; rs[threadIdx.x >> 5] = ss; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tw = 0.0, ts = 0.0;
    for (int w = 0; w < kInstThreads / 32; ++w) { tw += rw[w]; ts += rs[w]; }
    out[2 * i] = tw + ts;
    out[2 * i + 1] = tw;
  }
}

// Batches: scale both halves of instance i's entries of a vector by scale[i]
// (blockIdx.y = instance).  The vector is column *col + col_offset of v with
// stride ld (v itself if col is null); nothing is done when *skip != 0.
template <typename T>
__global__ void k_inst_scale(T* __restrict__ v, size_t half, const long long* __restrict__ range,
                             const double* __restrict__ scale, const int* col, int col_offset, size_t ld,
                             const int* skip) {
  if (skip && *skip) return;
  T* base = col ? v + size_t(*col + col_offset) * ld : v;
  const int i = blockIdx.y;
  const T sc = T(scale[i]);
  const long long a = range[2 * i], cnt = range[2 * i + 1];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < cnt; t += (long long)gridDim.x * blockDim.x) {
    base[a + t] *= sc;
    base[half + a + t] *= sc;
  }
}

}  // namespace hbpc

using namespace hbpc;

static thread_local std::string g_create_error;

struct hbpc_batch {
  std::vector<hbpc_ctx*> g;       // groups (one per N)
  std::vector<int> ig, il;        // instance -> group, index within the group
  std::string err;
};

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
  // BR2 viscous term: derivative tables (FP64 and FP32) and element blocks
  double* vtab_d = nullptr;
  float* vtab_f = nullptr;
  double* vloc_d = nullptr;
  // batch of instances sharing N (hbpc_batch_*); ninst = 0 for one problem
  int ninst = 0;
  std::vector<long long> ie0, inE;         // element range of every instance
  std::vector<hbpc_mesh> imesh;
  std::vector<double> inu;
  InstGeo<double>* d_inst = nullptr;
  InstGeo<float>* d_instf = nullptr;
  int* d_blk = nullptr;                    // operator block -> instance
  long long* d_irange = nullptr;           // per instance: first value, count (one half)
  double* d_inrm = nullptr;                // per-instance squared norms
  double* d_iscale = nullptr;              // per-instance row scaling of the GMRES system
  std::vector<double> h_iscale;
  // per-instance GMRES of the mixed mode (batch_krylov.cuh)
  bool bk = false;
  int bk_grid = 0;
  BKrylovT<float> BK{};
  void* bk_mem = nullptr;                  // one allocation for all of BK's device arrays
  std::vector<double> h_inrm;
  std::vector<int> h_active;
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
  // 1: the block preconditioner is rebuilt before every Newton iteration (the
  // setting of the paper's study, Sec. 4.1.2); 0: once per Newton solve, at
  // its first iterate (the reuse the paper suggests, end of Sec. 4.1.2)
  int pc_every = 1;
  // BJ_ext with one block for all elements: linear advection (with or without
  // a viscous term) on one uniform mesh has the same J_i in every element and
  // for every state, so one J, one S^-1 serve the whole mesh
  bool pc_shared = false;
  // some direction has boundaries (hbpc_set_boundary): the element blocks of a
  // linear problem then differ at the boundary elements
  bool bounded = false;
  // BJ^H_ext with a nonlinear flux: the Hessian blocks are in M (pc_build)
  // and the apply takes the BJ^H_ext algebra
  bool pc_hess = false;
  double pc_c1 = 0.0, pc_c2 = 0.0;
  // the shared block's J as 1-D Kronecker factors (k_pc_kron_factors)
  double* kron_d = nullptr;
  float* kron_f = nullptr;
  int* kron_ok = nullptr;
  // the shared FP64 block's apply on the tensor cores (bjext_tc.cuh): P's
  // digit planes and row exponents, formed at every build; ptc_ready when
  // they match the current blocks; HBPC_PC_TC=0 keeps the CUDA-core apply
  __nv_bfloat16* ptc_planes = nullptr;
  int* ptc_exp = nullptr;
  int* ptc_err = nullptr;
  bool ptc_ready = false;
  int ptc_enable = 1;
  // mixed precision (FP32 Krylov loop, FP64 Newton)
  DGParams<float> prmf{};
  KrylovT<float> Kf{};
  float* Vf = nullptr;      // FP32 Krylov basis
  float* Zf = nullptr;      // FP32 preconditioned vector / scratch, 2 n_dof
  float* Zf2 = nullptr;     // FP32 scratch, 2 n_dof
  float* Wf = nullptr;      // FP32 copy of the linearisation point (W, sigma)
  float* Mf = nullptr;      // FP32 copies of the BJ_ext blocks
  float* Jf = nullptr;
  // learned block preconditioner (network, replay buffer, scratch)
  struct Learned {
    bool alloc = false;
    int nb = 0, din = 0, dinp = 0, H = kMlpHidden, dout = 0, doutp = 0;
    size_t np = 0, np_train = 0, oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
    float* P = nullptr; float* G = nullptr; float* Mo = nullptr; float* Ve = nullptr;
    __nv_bfloat16* W1h = nullptr; __nv_bfloat16* W2h = nullptr; __nv_bfloat16* W3h = nullptr;
    __nv_bfloat16* W2T = nullptr; __nv_bfloat16* W3T = nullptr;
    __nv_bfloat16* W3p = nullptr;   // W3's rows in block storage order (inference)
    float* bp = nullptr;            // per class: bias + class mean + identity in storage order
    float* mu = nullptr; float* sd = nullptr;
    float* ckey = nullptr; float* cmean = nullptr;   // stage classes and their mean inverses
    int* vflag = nullptr;                             // per element: learned block failed its check
    int* vcount = nullptr;                            // blocks replaced by the exact inverse (running sum)
    int* gerr = nullptr;                              // a tensor-core GEMM's bounded wait ran out
    unsigned long long builds = 0;
    int* cls = nullptr;                               // class of every training sample
    bool stats = false;
    int adam_t = 0;
    int cap = 0, count = 0, next = 0, per_newton = 0, offset = 0;
    float* featbuf = nullptr; float* Jbuf = nullptr; float* cbuf = nullptr;
    float* Tbuf = nullptr;          // exact block inverses of the BJ_ext path (targets)
    bool targets = true;            // every collected row has a target
    int last_off = 0, last_row = 0, last_count = 0;
    __nv_bfloat16* Fi = nullptr; __nv_bfloat16* H1i = nullptr; __nv_bfloat16* H2i = nullptr;
    int Bmax = 0;
    __nv_bfloat16 *Fb = nullptr, *H1b = nullptr, *H2b = nullptr, *dOb = nullptr, *dZ2 = nullptr, *dZ1 = nullptr;
    __nv_bfloat16 *dOT = nullptr, *H2T = nullptr, *dZ2T = nullptr, *H1T = nullptr, *dZ1T = nullptr, *FT = nullptr;
    float *Jb = nullptr, *cb = nullptr, *Ob = nullptr, *Xb = nullptr;
    double* lpart = nullptr;
    int* idx = nullptr;
  } lp;
  Krylov K{};
  hbpc_stats stats{};
  std::string err;
  int nblocks = 0;
  int vcount_base = 0;      // learned-block fallbacks before the last reset_stats
  int vcols = 0;            // columns of the FP64 basis V
  bool coop = false;        // CGS2 as one cooperative launch (all blocks resident)
  int coop_max_blocks = 0;  // resident blocks of the cooperative kernel
  int sms = 0;
  int verbose = 0;          // HBPC_VERBOSE=1: Newton/GMRES trace on stderr
  // CUDA graphs of one batch of Arnoldi steps ([0] FP64, [1] mixed); graph_mode
  // 0 (HBPC_GRAPH=0) launches the kernels one by one
  struct ArnGraph {
    cudaGraphExec_t exec = nullptr;
    bool failed = false;        // the runtime refused the capture: direct launches
    long long launches = 0;     // kernel launches the graph replays
    long long key[8] = {};      // launch shapes it was captured with
  } arn_graph[3];   // [2]: the Schur form
  int graph_mode = 1;
  // the device-driven step (hbpc_set_step_graph): one CUDA graph per HBPC step,
  // its Newton and GMRES loops as conditional WHILE/IF nodes
  struct StepGraph {
    bool on = false;
    bool capturing = false;              // the step is being captured (no host waits)
    cudaGraphExec_t exec = nullptr;
    std::vector<unsigned char> key;      // configuration the graph was built for
    cudaStream_t cap = nullptr;          // stream the graph is captured on
    StepCtl* ctl = nullptr;              // device control block
    StepCtl* ctl_host = nullptr;         // pinned copy, read after the graph
    double* g0 = nullptr;                // per instance (groups): ||G_i^0||, ||dW_i||, active
    double* dw = nullptr;
    int* active = nullptr;
    long long top_launches = 0, top_r1 = 0, top_r2 = 0;   // per step, outside the loops
  } sg;
  double wait_limit_s = 0.0;  // bounded host waits (hbpc_set_wait_limit); 0 = none
  // every instance of a batch group has the same mesh (then J_i is shared
  // between instances as between elements)
  bool same_mesh = false;
  // corrector batching: the s - 1 corrector stages of a sweep as the
  // instances of one group context (hbpc_set_corrector_batch), on this stream
  hbpc_ctx* cb = nullptr;
  // Schur form of the Newton systems (hbpc_set_schur): scratch 2 n vectors,
  // the right-hand side and the norms of the product inputs
  bool schur = false;
  double* sa = nullptr;
  double* sb = nullptr;
  double* srhs = nullptr;
  double* snrm = nullptr;   // 3 norms (total, W, sigma) of the current product input
  Prof prof;
};

namespace {

constexpr int kMaxPcBlock = 160;   // largest BJ_ext block (shared-memory inverse)
// A learned block M~ is kept when |M~ S x - x| <= tau |x| for a random sign
// probe x; otherwise the element gets the exact inverse.
constexpr double kPcVerifyTau = 0.5;

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

// Wait for the context's stream.  With a wait limit the stream is polled and
// the wait gives up with HBPC_ERR_TIMEOUT after that many seconds (the work
// keeps running on the device).
hbpc_status sync(hbpc_ctx* x, const char* where) {
  cudaError_t e = cudaSuccess;
  if (x->wait_limit_s > 0.0) {
    const auto t0 = std::chrono::steady_clock::now();
    for (long long spin = 0;; ++spin) {
      e = cudaStreamQuery(x->stream);
      if (e != cudaErrorNotReady) break;
      const double waited = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (waited > x->wait_limit_s)
        return fail(x, HBPC_ERR_TIMEOUT, std::string(where) + ": the wait limit ran out");
      if (spin > 64) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  } else {
    e = cudaStreamSynchronize(x->stream);
  }
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
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_norms<double, double><<<x->nblocks, kVecThreads, 0, x->stream>>>(v, n, size_t(x->ndof), x->K, nullptr));
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
  if (x->sol.pc != HBPC_PC_NONE) {   // Jv acts on z = P^-1 v_j, kept in Z
    z.V = x->Z; z.jidx = nullptr; z.vscale = nullptr;
    z.nrmW = x->zn + 1; z.nrmS = x->zn + 2;
  }
  return z;
}

// The shared-block apply (k_pc_apply_shared, 2 elements per thread) when its
// shared memory fits the default 48 KB and no norms are wanted; false: the
// caller launches the general apply (which also handles a shared block).
constexpr int kPcSharedEG = 2;
template <typename S>
bool pc_shared_launch(hbpc_ctx* x, const PcApplyT<S>& a) {
  if (a.zn) return false;
  const int nb = a.nb;
  const int groups = 256 / nb;
  if (groups < 1) return false;
  const size_t smem = (2 * size_t(nb) * nb + 4 * size_t(kPcSharedEG) * nb * groups) * sizeof(S);
  if (smem > 48 * 1024) return false;
  const int per_block = groups * kPcSharedEG;
  const int grid = int((x->nE + per_block - 1) / per_block);
  HBPC_RUN(x, HBPC_PHASE_PC, 1,
           (k_pc_apply_shared<S, kPcSharedEG><<<grid, groups * nb, smem, x->stream>>>(a)));
  return cudaPeekAtLastError() == cudaSuccess;
}

// P^-1 applied to scale * in -> out (out += when accumulate), norms to x->zn
hbpc_status pc_apply(hbpc_ctx* x, const double* in, const int* jidx, const double* scale,
                     double* out, int accumulate, const int* skip) {
  PcApply a{};
  a.M = x->Mpc; a.J = x->Jpc;
  a.xW = in; a.xS = in + x->ndof;
  a.scale = scale; a.jidx = jidx; a.ld = size_t(2 * x->ndof);
  a.oW = out; a.oS = out + x->ndof;
  a.c12 = x->c12; a.skip = skip; a.accumulate = accumulate;
  a.zn = x->ops.jv_linear ? nullptr : x->zn;   // ||z|| halves feed eps_FD of Eq. 23 only
  a.nb = x->nb; a.nE = int(x->nE);
  a.shared = x->pc_shared ? 1 : 0;
  a.kron = x->pc_shared ? x->kron_d : nullptr; a.kron_ok = x->kron_ok; a.P = x->P; a.dim = x->dim;
  a.hess = x->pc_hess ? 1 : 0;
  if (a.shared && !a.hess && !a.zn && x->ptc_ready) {
    PcApplyTc t{};
    t.planes = x->ptc_planes; t.pexp = x->ptc_exp;
    t.xW = a.xW; t.xS = a.xS; t.scale = scale; t.jidx = jidx; t.ld = a.ld;
    t.oW = a.oW; t.oS = a.oS; t.skip = skip; t.accumulate = accumulate;
    t.nb = x->nb; t.nE = int(x->nE); t.err = x->ptc_err;
    const int grid = int((x->nE + kPtcElems - 1) / kPtcElems);
    HBPC_RUN(x, HBPC_PHASE_PC, 1,
             k_pc_apply_tc<<<grid, kPtcThreads, PtcDims(x->nb).smem(), x->stream>>>(t));
    HBPC_LAUNCH_CK(x, "k_pc_apply_tc");
    return HBPC_OK;
  }
  if (a.shared && pc_shared_launch(x, a)) return HBPC_OK;
  HBPC_RUN(x, HBPC_PHASE_PC, 1, k_pc_apply<double><<<x->pc_grid, x->pc_threads, x->pc_smem, x->stream>>>(a, x->K));
  HBPC_LAUNCH_CK(x, "k_pc_apply");
  return HBPC_OK;
}

// FP32 version for the mixed mode (blocks in Mf, Jf)
hbpc_status pc_apply_f(hbpc_ctx* x, const float* in, const int* jidx, const double* scale, float* out,
                       int accumulate, const int* skip) {
  PcApplyT<float> a{};
  a.M = x->Mf; a.J = x->Jf;
  a.xW = in; a.xS = in + x->ndof;
  a.scale = scale; a.jidx = jidx; a.ld = size_t(2 * x->ndof);
  a.oW = out; a.oS = out + x->ndof;
  a.c12 = x->c12; a.skip = skip; a.accumulate = accumulate;
  a.zn = nullptr;   // the analytic FP32 Jv needs no norms
  a.nb = x->nb; a.nE = int(x->nE);
  a.shared = x->pc_shared ? 1 : 0;
  a.kron = x->pc_shared ? x->kron_f : nullptr; a.kron_ok = x->kron_ok; a.P = x->P; a.dim = x->dim;
  a.hess = x->pc_hess ? 1 : 0;
  if (a.shared && pc_shared_launch(x, a)) return HBPC_OK;
  HBPC_RUN(x, HBPC_PHASE_PC, 1, k_pc_apply<float><<<x->pc_grid, x->pc_threads, x->pc_smem, x->stream>>>(a, x->K));
  HBPC_LAUNCH_CK(x, "k_pc_apply<float>");
  return HBPC_OK;
}

hbpc_status to_float(hbpc_ctx* x, const double* in, float* out, size_t n) {
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_to_float<<<grid_for(n), 256, 0, x->stream>>>(in, out, n, 1.0));
  HBPC_LAUNCH_CK(x, "k_to_float");
  return HBPC_OK;
}

// ---------------------------------------------------------------------------
// Learned block preconditioner (mlp.cuh): allocation, inference, training.
// ---------------------------------------------------------------------------
template <typename Tp>
hbpc_status dalloc_any(hbpc_ctx* x, Tp** p, size_t count) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(Tp));
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(x, HBPC_ERR_OOM, std::string("cudaMalloc (learned preconditioner): ") + cudaGetErrorString(e));
  }
  return HBPC_OK;
}

template <class Epi>
hbpc_status gemm(hbpc_ctx* x, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N,
                 int K, Epi epi) {
  if (K % 8 || lda % 8 || ldb % 8 || (reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15))
    return fail(x, HBPC_ERR_INVALID_ARG, "GEMM operands must be 16-byte aligned with K, ld multiples of 8");
  if (M <= 0 || N <= 0 || K <= 0) return HBPC_OK;
  static const cudaError_t attr =
      cudaFuncSetAttribute(k_gemm_bf16_tc<Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
  if (attr != cudaSuccess) return cuda_fail(x, attr, "tensor-core GEMM shared memory");
  CUtensorMap ta, tb;
  if (!tc_tensor_map(&ta, A, K, M, lda) || !tc_tensor_map(&tb, B, K, N, ldb))
    return fail(x, HBPC_ERR_CUDA, "tensor map of a GEMM operand rejected");
  const dim3 grid((N + kTcBN - 1) / kTcBN, (M + kTcBM - 1) / kTcBM);
  HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1, k_gemm_bf16_tc<Epi><<<grid, kTcThreads, kTcSmem, x->stream>>>(ta, tb, M, N, K, epi, x->lp.gerr));
  HBPC_LAUNCH_CK(x, "k_gemm_bf16_tc");
  return HBPC_OK;
}

hbpc_status lp_transpose(hbpc_ctx* x, const __nv_bfloat16* in, __nv_bfloat16* out, int rows, int cols) {
  const dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
  HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1, k_transpose_bf16<<<grid, block, 0, x->stream>>>(in, out, rows, cols));
  HBPC_LAUNCH_CK(x, "k_transpose_bf16");
  return HBPC_OK;
}

// Allocate the network, its optimiser state and the inference scratch.
hbpc_status lp_alloc(hbpc_ctx* x) {
  auto& L = x->lp;
  if (L.alloc) return HBPC_OK;
  L.nb = x->nb;
  L.din = L.nb + 2;
  L.dinp = ((L.din + 15) / 16) * 16;
  L.dout = L.nb * L.nb;
  L.doutp = ((L.dout + 7) / 8) * 8;
  const size_t H = size_t(L.H);
  L.oW1 = 0; L.ob1 = L.oW1 + H * L.dinp; L.oW2 = L.ob1 + H; L.ob2 = L.oW2 + H * H;
  L.oW3 = L.ob2 + H; L.ob3 = L.oW3 + size_t(L.doutp) * H; L.np_train = L.ob3 + L.doutp;
  // + feature standardisation (mu, sd), stage-class keys and mean inverses
  L.np = L.np_train + 2 * size_t(L.dinp) + 2 * kMlpClasses + size_t(kMlpClasses) * L.doutp;
  hbpc_status e;
  if ((e = dalloc_any(x, &L.P, L.np)) || (e = dalloc_any(x, &L.G, L.np)) || (e = dalloc_any(x, &L.Mo, L.np)) ||
      (e = dalloc_any(x, &L.Ve, L.np)) || (e = dalloc_any(x, &L.W1h, H * L.dinp)) ||
      (e = dalloc_any(x, &L.W2h, H * H)) || (e = dalloc_any(x, &L.W3h, size_t(L.doutp) * H)) ||
      (e = dalloc_any(x, &L.W2T, H * H)) || (e = dalloc_any(x, &L.W3T, size_t(L.doutp) * H)) ||
      (e = dalloc_any(x, &L.W3p, size_t(L.doutp) * H)) || (e = dalloc_any(x, &L.bp, size_t(kMlpClasses) * L.doutp)) ||
      (e = dalloc_any(x, &L.Fi, size_t(x->nE) * L.dinp)) || (e = dalloc_any(x, &L.H1i, size_t(x->nE) * H)) ||
      (e = dalloc_any(x, &L.H2i, size_t(x->nE) * H)))
    return e;
  if ((e = dalloc_any(x, &L.vflag, size_t(x->nE))) || (e = dalloc_any(x, &L.vcount, 1)) ||
      (e = dalloc_any(x, &L.gerr, 1)))
    return e;
  HBPC_CK(x, cudaMemsetAsync(L.vcount, 0, sizeof(int), x->stream));
  HBPC_CK(x, cudaMemsetAsync(L.gerr, 0, sizeof(int), x->stream));
  L.mu = L.P + L.np_train;
  L.sd = L.mu + L.dinp;
  L.ckey = L.sd + L.dinp;
  L.cmean = L.ckey + 2 * kMlpClasses;
  HBPC_CK(x, cudaMemsetAsync(L.P, 0, L.np * sizeof(float), x->stream));
  HBPC_CK(x, cudaMemsetAsync(L.Mo, 0, L.np * sizeof(float), x->stream));
  HBPC_CK(x, cudaMemsetAsync(L.Ve, 0, L.np * sizeof(float), x->stream));
  std::vector<float> ones(L.dinp, 1.0f);
  HBPC_CK(x, cudaStreamSynchronize(x->stream));
  HBPC_CK(x, cudaMemcpy(L.sd, ones.data(), L.dinp * sizeof(float), cudaMemcpyHostToDevice));
  L.alloc = true;
  return HBPC_OK;
}

hbpc_status lp_alloc_train(hbpc_ctx* x, int B, int P) {
  auto& L = x->lp;
  hbpc_status e;
  if ((e = lp_alloc(x)) != HBPC_OK) return e;
  if (B <= L.Bmax && L.Xb && P * L.nb * B <= L.Bmax * 16 * L.nb) return HBPC_OK;
  const size_t Bs = size_t(B), H = size_t(L.H);
  for (void* q : {(void*)L.Fb, (void*)L.H1b, (void*)L.H2b, (void*)L.dOb, (void*)L.dZ2, (void*)L.dZ1,
                  (void*)L.dOT, (void*)L.H2T, (void*)L.dZ2T, (void*)L.H1T, (void*)L.dZ1T, (void*)L.FT,
                  (void*)L.Jb, (void*)L.cb, (void*)L.Ob, (void*)L.Xb, (void*)L.lpart, (void*)L.idx, (void*)L.cls})
    cudaFree(q);
  if ((e = dalloc_any(x, &L.Fb, Bs * L.dinp)) || (e = dalloc_any(x, &L.H1b, Bs * H)) ||
      (e = dalloc_any(x, &L.H2b, Bs * H)) || (e = dalloc_any(x, &L.dOb, Bs * L.doutp)) ||
      (e = dalloc_any(x, &L.dZ2, Bs * H)) || (e = dalloc_any(x, &L.dZ1, Bs * H)) ||
      (e = dalloc_any(x, &L.dOT, Bs * L.doutp)) || (e = dalloc_any(x, &L.H2T, Bs * H)) ||
      (e = dalloc_any(x, &L.dZ2T, Bs * H)) || (e = dalloc_any(x, &L.H1T, Bs * H)) ||
      (e = dalloc_any(x, &L.dZ1T, Bs * H)) || (e = dalloc_any(x, &L.FT, Bs * L.dinp)) ||
      (e = dalloc_any(x, &L.Jb, Bs * L.dout)) || (e = dalloc_any(x, &L.cb, Bs * 2)) ||
      (e = dalloc_any(x, &L.Ob, Bs * L.doutp)) || (e = dalloc_any(x, &L.Xb, Bs * 16 * L.nb)) ||
      (e = dalloc_any(x, &L.lpart, Bs)) || (e = dalloc_any(x, &L.idx, Bs)) || (e = dalloc_any(x, &L.cls, Bs)))
    return e;
  HBPC_CK(x, cudaMemsetAsync(L.dOb, 0, Bs * L.doutp * sizeof(__nv_bfloat16), x->stream));
  L.Bmax = B;
  return HBPC_OK;
}

// The flag of the tensor-core GEMMs' bounded waits (read after the stream's
// work; a set flag is an error and is cleared).
hbpc_status lp_gemm_check(hbpc_ctx* x) {
  if (!x->lp.gerr) return HBPC_OK;
  int e = 0;
  HBPC_CK(x, cudaMemcpyAsync(&e, x->lp.gerr, sizeof(int), cudaMemcpyDeviceToHost, x->stream));
  hbpc_status s = sync(x, "tensor-core GEMM");
  if (s != HBPC_OK) return s;
  if (e) {
    HBPC_CK(x, cudaMemsetAsync(x->lp.gerr, 0, sizeof(int), x->stream));
    return fail(x, HBPC_ERR_CUDA, "a tensor-core GEMM gave up waiting for its MMAs");
  }
  return HBPC_OK;
}

// The flag of the tensor-core block apply's bounded waits (a wait that ran
// out wrote NaN outputs): read after the stream's work; a set flag is
// HBPC_ERR_TIMEOUT (with `what`) and is cleared.
hbpc_status ptc_check(hbpc_ctx* x, const std::string& what) {
  if (!x->ptc_err) return HBPC_OK;
  int e = 0;
  if (cudaMemcpyAsync(&e, x->ptc_err, sizeof(int), cudaMemcpyDeviceToHost, x->stream) != cudaSuccess ||
      cudaStreamSynchronize(x->stream) != cudaSuccess || !e)
    return HBPC_OK;
  cudaMemsetAsync(x->ptc_err, 0, sizeof(int), x->stream);
  return fail(x, HBPC_ERR_TIMEOUT, what + " (a bounded wait of the tensor-core block apply ran out)");
}

// A non-finite result: HBPC_ERR_TIMEOUT when the tensor-core block apply gave
// up waiting (its NaN outputs are the cause), else HBPC_ERR_NONFINITE.
hbpc_status nonfinite(hbpc_ctx* x, const std::string& what) {
  const hbpc_status t = ptc_check(x, what);
  return t != HBPC_OK ? t : fail(x, HBPC_ERR_NONFINITE, what);
}

void lp_free(hbpc_ctx* x) {
  auto& L = x->lp;
  for (void* q : {(void*)L.P, (void*)L.G, (void*)L.Mo, (void*)L.Ve, (void*)L.W1h, (void*)L.W2h, (void*)L.W3h,
                  (void*)L.W2T, (void*)L.W3T, (void*)L.featbuf, (void*)L.Jbuf, (void*)L.Tbuf,
                  (void*)L.cbuf, (void*)L.Fi, (void*)L.H1i, (void*)L.H2i, (void*)L.Fb, (void*)L.H1b, (void*)L.H2b,
                  (void*)L.dOb, (void*)L.dZ2, (void*)L.dZ1, (void*)L.dOT, (void*)L.H2T, (void*)L.dZ2T,
                  (void*)L.H1T, (void*)L.dZ1T, (void*)L.FT, (void*)L.Jb, (void*)L.cb, (void*)L.Ob, (void*)L.Xb,
                  (void*)L.lpart, (void*)L.idx, (void*)L.cls, (void*)L.vflag, (void*)L.vcount, (void*)L.gerr,
                  (void*)L.W3p, (void*)L.bp})
    cudaFree(q);
  L = hbpc_ctx::Learned{};
}

// BF16 copies of the weights (and the transposes used by the backward pass)
hbpc_status lp_refresh(hbpc_ctx* x) {
  auto& L = x->lp;
  const size_t H = size_t(L.H);
  HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1, k_f32_to_bf16<<<grid_for(H * L.dinp), 256, 0, x->stream>>>(L.P + L.oW1, L.W1h, H * L.dinp));
  HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1, k_f32_to_bf16<<<grid_for(H * H), 256, 0, x->stream>>>(L.P + L.oW2, L.W2h, H * H));
  HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1, k_f32_to_bf16<<<grid_for(size_t(L.doutp) * H), 256, 0, x->stream>>>(L.P + L.oW3, L.W3h, size_t(L.doutp) * H));
  HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1, k_w3_permute<<<grid_for(size_t(L.doutp) * H), 256, 0, x->stream>>>(L.W3h, L.W3p, L.nb, L.doutp, L.H));
  HBPC_LAUNCH_CK(x, "lp_refresh");
  hbpc_status s;
  if ((s = lp_transpose(x, L.W2h, L.W2T, L.H, L.H)) != HBPC_OK) return s;
  return lp_transpose(x, L.W3h, L.W3T, L.doutp, L.H);
}

// M~_e for every element from the current network (replaces the LU of BJ_ext).
hbpc_status lp_infer(hbpc_ctx* x, const double* W, double c1, double c2) {
  auto& L = x->lp;
  if (!L.alloc) return fail(x, HBPC_ERR_INVALID_ARG, "learned preconditioner has no network");
  hbpc_status s;
  const size_t nf = size_t(x->nE) * L.dinp;
  HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1, k_mlp_features<<<grid_for(nf), 256, 0, x->stream>>>(W, int(x->nE), L.nb, c1, c2, L.mu, L.sd, L.dinp, L.Fi));
  HBPC_LAUNCH_CK(x, "k_mlp_features");
  const int nE = int(x->nE);
  if ((s = gemm(x, L.Fi, L.dinp, L.W1h, L.dinp, nE, L.H, L.dinp, EpiBiasTanh{L.P + L.ob1, L.H1i, L.H})) != HBPC_OK) return s;
  if ((s = gemm(x, L.H1i, L.H, L.W2h, L.H, nE, L.H, L.H, EpiBiasTanh{L.P + L.ob2, L.H2i, L.H})) != HBPC_OK) return s;
  // the stage class of (c1, c2) from the keys (host copy of the parameters' keys)
  float keys[2 * kMlpClasses];
  HBPC_CK(x, cudaMemcpyAsync(keys, L.ckey, sizeof(keys), cudaMemcpyDeviceToHost, x->stream));
  if ((s = lp_gemm_check(x)) != HBPC_OK) return s;   // waits for the keys too
  const float* cm = L.cmean + size_t(mlp_class(keys, float(c1), float(c2))) * L.doutp;
  HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1, k_pc_bias_storage<<<grid_for(L.doutp), 256, 0, x->stream>>>(L.P + L.ob3, cm, 1, L.nb, L.doutp, L.bp));
  if (x->sol.precision == HBPC_PREC_MIXED)
    return gemm(x, L.H2i, L.H, L.W3p, L.H, nE, L.dout, L.H, EpiPcBlock<float>{L.bp, nullptr, L.doutp, x->Mf, L.nb});
  return gemm(x, L.H2i, L.H, L.W3p, L.H, nE, L.dout, L.H, EpiPcBlock<double>{L.bp, nullptr, L.doutp, x->Mpc, L.nb});
}

// One forward/backward pass on the batch already in Fb, Jb, cb, Xb: loss and
// gradients (in L.G).
hbpc_status lp_loss_grad(hbpc_ctx* x, int B, int P, double* loss, int kind) {
  auto& L = x->lp;
  hbpc_status s;
  const int H = L.H;
  // forward
  if ((s = gemm(x, L.Fb, L.dinp, L.W1h, L.dinp, B, H, L.dinp, EpiBiasTanh{L.P + L.ob1, L.H1b, H})) != HBPC_OK) return s;
  if ((s = gemm(x, L.H1b, H, L.W2h, H, B, H, H, EpiBiasTanh{L.P + L.ob2, L.H2b, H})) != HBPC_OK) return s;
  if ((s = gemm(x, L.H2b, H, L.W3h, H, B, L.doutp, H, EpiBiasF32{L.P + L.ob3, L.Ob, L.doutp})) != HBPC_OK) return s;
  // loss and dO (dO keeps the n_b^2-wide row layout inside its doutp-wide rows);
  // Jb holds J (probe loss) or the target inverse (inverse regression)
  HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1, k_mlp_classify<<<(B + 255) / 256, 256, 0, x->stream>>>(L.cb, B, L.ckey, L.cls));
  if (kind == HBPC_PC_LOSS_INVERSE) {
    HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1, k_mlp_inverse_loss<<<B, 256, 0, x->stream>>>(L.Jb, L.Ob, B, L.nb, L.doutp, L.cmean, L.cls, L.dOb, L.lpart));
    HBPC_LAUNCH_CK(x, "k_mlp_inverse_loss");
  } else {
    const size_t shm = size_t(2 * P + 2) * L.nb * sizeof(float);
    HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1, k_mlp_probe_loss<<<B, 256, shm, x->stream>>>(L.Jb, L.cb, L.Ob, L.Xb, B, P, L.nb, L.doutp, L.cmean, L.cls, L.dOb, L.lpart));
    HBPC_LAUNCH_CK(x, "k_mlp_probe_loss");
  }
  // backward: W3, b3
  if ((s = lp_transpose(x, L.dOb, L.dOT, B, L.doutp)) != HBPC_OK) return s;
  if ((s = lp_transpose(x, L.H2b, L.H2T, B, H)) != HBPC_OK) return s;
  if ((s = gemm(x, L.dOT, B, L.H2T, B, L.doutp, H, B, EpiStore{L.G + L.oW3, H})) != HBPC_OK) return s;
  HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1, k_colsum_bf16<<<(L.doutp + 255) / 256, 256, 0, x->stream>>>(L.dOb, B, L.doutp, L.G + L.ob3));
  // dZ2 = (dO W3) * (1 - h2^2)
  if ((s = gemm(x, L.dOb, L.doutp, L.W3T, L.doutp, B, H, L.doutp, EpiDtanh{L.H2b, L.dZ2, H})) != HBPC_OK) return s;
  if ((s = lp_transpose(x, L.dZ2, L.dZ2T, B, H)) != HBPC_OK) return s;
  if ((s = lp_transpose(x, L.H1b, L.H1T, B, H)) != HBPC_OK) return s;
  if ((s = gemm(x, L.dZ2T, B, L.H1T, B, H, H, B, EpiStore{L.G + L.oW2, H})) != HBPC_OK) return s;
  HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1, k_colsum_bf16<<<(H + 255) / 256, 256, 0, x->stream>>>(L.dZ2, B, H, L.G + L.ob2));
  // dZ1 = (dZ2 W2) * (1 - h1^2)
  if ((s = gemm(x, L.dZ2, H, L.W2T, H, B, H, H, EpiDtanh{L.H1b, L.dZ1, H})) != HBPC_OK) return s;
  if ((s = lp_transpose(x, L.dZ1, L.dZ1T, B, H)) != HBPC_OK) return s;
  if ((s = lp_transpose(x, L.Fb, L.FT, B, L.dinp)) != HBPC_OK) return s;
  if ((s = gemm(x, L.dZ1T, B, L.FT, B, H, L.dinp, B, EpiStore{L.G + L.oW1, L.dinp})) != HBPC_OK) return s;
  HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1, k_colsum_bf16<<<(H + 255) / 256, 256, 0, x->stream>>>(L.dZ1, B, H, L.G + L.ob1));
  HBPC_LAUNCH_CK(x, "lp backward");
  if (loss) {
    std::vector<double> lp(B);
    HBPC_CK(x, cudaMemcpyAsync(lp.data(), L.lpart, B * sizeof(double), cudaMemcpyDeviceToHost, x->stream));
    if ((s = sync(x, "lp loss")) != HBPC_OK) return s;
    double t = 0.0;
    for (int i = 0; i < B; ++i) t += lp[i];
    *loss = t;
  }
  return HBPC_OK;
}

// Sample the current Newton iteration's element Jacobians into the replay buffer.
hbpc_status lp_collect(hbpc_ctx* x, const double* W, double c1, double c2) {
  auto& L = x->lp;
  if (L.per_newton <= 0 || !L.featbuf) return HBPC_OK;
  const int count = std::min<int>(L.per_newton, int(x->nE));
  const int stride = std::max<int>(1, int(x->nE) / count);
  HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1,
           x->sol.precision == HBPC_PREC_MIXED
               ? k_mlp_collect<float><<<count, 128, 0, x->stream>>>(W, x->Jf, int(x->nE), L.nb, c1, c2, count,
                                                                     stride, L.offset, L.next, L.cap, L.featbuf,
                                                                     L.Jbuf, L.cbuf)
               : k_mlp_collect<double><<<count, 128, 0, x->stream>>>(W, x->Jpc, int(x->nE), L.nb, c1, c2, count,
                                                                      stride, L.offset, L.next, L.cap, L.featbuf,
                                                                      L.Jbuf, L.cbuf));
  HBPC_LAUNCH_CK(x, "k_mlp_collect");
  L.last_off = L.offset; L.last_row = L.next; L.last_count = count;
  L.offset = (L.offset + 1) % std::max(1, stride);
  L.next = (L.next + count) % L.cap;
  L.count = std::min(L.cap, L.count + count);
  return HBPC_OK;
}

// Build J_i, S_i and M_i = S_i^-1 at the state W for the current c1, c2.
hbpc_status pc_build(hbpc_ctx* x, const double* W, double c1, double c2) {
  const bool linear = x->phys.law == HBPC_LAW_ADVECTION;
  const bool collecting = x->lp.per_newton > 0;
  // (a captured step rebuilds every time: its replays do not see this test)
  if (!x->sg.capturing && linear && !collecting && x->sol.pc != HBPC_PC_LEARNED && x->pc_built &&
      x->pc_c1 == c1 && x->pc_c2 == c2)
    return HBPC_OK;
  const size_t nb = size_t(x->nb);
  const bool mixed = x->sol.precision == HBPC_PREC_MIXED;
  // one shared block when J_i is the same for every element and state (the
  // training-data collection and the learned network want per-element blocks)
  x->pc_shared = linear && !x->bounded && (x->ninst == 0 || x->same_mesh) &&
                 (x->sol.pc == HBPC_PC_BJEXT || x->sol.pc == HBPC_PC_BJEXT_H) && !collecting;
  // BJ^H_ext: the Hessian blocks at (W, sigma), sigma the second half of the
  // extended state W points to; a linear flux has none (H = 0, Sec. 3.2.1)
  // and BJ^H_ext is then BJ_ext
  x->pc_hess = x->sol.pc == HBPC_PC_BJEXT_H && x->ops.pc_hessian != nullptr;
  const int nEb = x->pc_shared ? 1 : int(x->nE);   // blocks to build
  // J_i in the precision of the apply: FP32 in the mixed mode (the blocks only
  // precondition the FP32 Krylov loop), FP64 otherwise; the Hessian blocks go
  // straight into M, where S = I - c1 J + c2 (H + J^2) replaces them
  if (mixed) {
    DGParams<float> pf = x->prmf;
    pf.nE = nEb;
    HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1, x->ops.pc_assemble_f(pf, W, x->Jf, x->stream));
    if (x->pc_hess) HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1, x->ops.pc_hessian_f(pf, W, W + x->ndof, x->Mf, x->stream));
  } else {
    DGParams<double> pd = x->prm;
    pd.nE = nEb;
    HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1, x->ops.pc_assemble(pd, W, x->Jpc, x->stream));
    if (x->pc_hess) HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1, x->ops.pc_hessian(pd, W, W + x->ndof, x->Mpc, x->stream));
  }
  hbpc_status s0;
  if (collecting && (s0 = lp_collect(x, W, c1, c2)) != HBPC_OK) return s0;
  if (x->sol.pc == HBPC_PC_LEARNED) {   // M~ from the network instead of the LU
    if (collecting) x->lp.targets = false;   // no exact inverse for these rows
    if ((s0 = lp_infer(x, W, c1, c2)) != HBPC_OK) return s0;
    // check every learned block with a random probe; the blocks that fail get
    // the exact inverse (form S, Gauss-Jordan) instead
    auto& L = x->lp;
    const int epb = x->pc_threads / x->nb;
    const unsigned long long seed = 0x5EED0000ull + (L.builds++);
    if (mixed) {
      HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1,
               k_pc_verify<float><<<x->pc_grid, x->pc_threads, size_t(epb) * 3 * nb * sizeof(float), x->stream>>>(
                   x->Mf, x->Jf, x->nb, int(x->nE), x->c12, seed, kPcVerifyTau, L.vflag, L.vcount));
      HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1,
               k_pc_form_S<float><<<int(x->nE), 256, nb * nb * sizeof(float), x->stream>>>(x->Jf, x->Mf, x->nb,
                                                                                           int(x->nE), x->c12, L.vflag));
      HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1,
               k_pc_invert<float><<<int(x->nE), 256, (nb * nb + nb) * sizeof(float) + nb * sizeof(int), x->stream>>>(
                   x->Mf, x->nb, int(x->nE), x->singular, L.vflag));
    } else {
      HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1,
               k_pc_verify<double><<<x->pc_grid, x->pc_threads, size_t(epb) * 3 * nb * sizeof(double), x->stream>>>(
                   x->Mpc, x->Jpc, x->nb, int(x->nE), x->c12, seed, kPcVerifyTau, L.vflag, L.vcount));
      HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1,
               k_pc_form_S<double><<<int(x->nE), 256, nb * nb * sizeof(double), x->stream>>>(x->Jpc, x->Mpc, x->nb,
                                                                                             int(x->nE), x->c12, L.vflag));
      HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1,
               k_pc_invert<double><<<int(x->nE), 256, (nb * nb + nb) * sizeof(double) + nb * sizeof(int), x->stream>>>(
                   x->Mpc, x->nb, int(x->nE), x->singular, L.vflag));
    }
    HBPC_LAUNCH_CK(x, "learned block check");
    x->pc_built = true;
    x->pc_c1 = c1;
    x->pc_c2 = c2;
    return HBPC_OK;
  }
  if (mixed) {
    // S and its inverse in FP32 as well
    HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1,
             k_pc_form_S<float><<<nEb, 256, nb * nb * sizeof(float), x->stream>>>(x->Jf, x->Mf, x->nb, nEb, x->c12,
                                                                                 nullptr, x->pc_hess ? x->Mf : nullptr));
    HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1,
             k_pc_invert<float><<<nEb, 256, (nb * nb + nb) * sizeof(float) + nb * sizeof(int), x->stream>>>(
                 x->Mf, x->nb, nEb, x->singular));
  } else {
    HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1,
             k_pc_form_S<double><<<nEb, 256, nb * nb * sizeof(double), x->stream>>>(
                 x->Jpc, x->Mpc, x->nb, nEb, x->c12, nullptr, x->pc_hess ? x->Mpc : nullptr));
    HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1,
             k_pc_invert<double><<<nEb, 256, (nb * nb + nb) * sizeof(double) + nb * sizeof(int), x->stream>>>(
                 x->Mpc, x->nb, nEb, x->singular));
  }
  // the shared FP64 block's P = [[M, -c2 J M], [J M, M - c1 J M]] as digit
  // planes for the tensor-core apply
  x->ptc_ready = false;
  if (x->pc_shared && !mixed && !x->pc_hess && x->ptc_planes) {
    const PtcDims D(x->nb);
    HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1,
             k_pc_tc_planes<<<D.R, 128, 3 * nb * sizeof(double), x->stream>>>(x->Mpc, x->Jpc, x->nb, x->c12,
                                                                             x->ptc_planes, x->ptc_exp));
    x->ptc_ready = true;
  }
  if (x->pc_shared && x->kron_ok) {
    // the shared J_0 as Kronecker factors for the apply (checked entry by entry)
    int nn = 1;
    for (int m = 0; m < x->dim; ++m) nn *= x->P;
    if (nn == x->nb && x->P <= kMaxP) {
      if (mixed)
        HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1,
                 k_pc_kron_factors<float><<<1, 256, 0, x->stream>>>(x->Jf, x->nb, x->P, x->dim, 1e-5f, x->kron_f,
                                                                    x->kron_ok));
      else
        HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1,
                 k_pc_kron_factors<double><<<1, 256, 0, x->stream>>>(x->Jpc, x->nb, x->P, x->dim, 1e-12, x->kron_d,
                                                                     x->kron_ok));
    } else {
      HBPC_CK(x, cudaMemsetAsync(x->kron_ok, 0, sizeof(int), x->stream));
    }
  }
  if (collecting && x->lp.Tbuf) {   // the block inverses as training targets
    auto& L = x->lp;
    const int stride = std::max<int>(1, int(x->nE) / std::max(1, L.last_count));
    if (mixed)
      HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1,
               k_mlp_collect_target<float><<<L.last_count, 128, 0, x->stream>>>(
                   x->Mf, int(x->nE), L.nb, L.last_count, stride, L.last_off, L.last_row, L.cap, L.Tbuf));
    else
      HBPC_RUN(x, HBPC_PHASE_PC_BUILD, 1,
               k_mlp_collect_target<double><<<L.last_count, 128, 0, x->stream>>>(
                   x->Mpc, int(x->nE), L.nb, L.last_count, stride, L.last_off, L.last_row, L.cap, L.Tbuf));
  }
  HBPC_LAUNCH_CK(x, "pc build");
  if (x->sg.capturing) {   // the singular flag is read after the step graph
    x->pc_built = false;
    return HBPC_OK;
  }
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

// The four launches of one Gram-Schmidt (CGS2) column: dot, update + second
// dot, update + norms, finalisation (krylov.cuh).
template <typename S>
void cgs_launch(hbpc_ctx* x, const KrylovT<S>& K) {
  if (x->coop) {   // one cooperative launch (k_cgs_lowsync) instead of four
    const size_t shm = cgs_lowsync_smem<S>(K.m);
    // the halves' norms of the new column feed only the difference-quotient
    // Jv applied to the basis itself (FP64, nonlinear flux, no preconditioner)
    int half_norms = (!x->ops.jv_linear && x->sol.pc == HBPC_PC_NONE &&
                      x->sol.precision != HBPC_PREC_MIXED) ? 1 : 0;
    void* args[] = {const_cast<KrylovT<S>*>(&K), &half_norms};
    HBPC_RUN(x, HBPC_PHASE_DOT, 1,
             cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_cgs_lowsync<S>), dim3(x->nblocks),
                                         dim3(kVecThreads), args, shm, x->stream));
    return;
  }
  const size_t m1 = size_t(K.m + 1);
  HBPC_RUN(x, HBPC_PHASE_DOT, 1, k_cgs_dot<S><<<x->nblocks, kVecThreads, m1 * kVecWarps * sizeof(double), x->stream>>>(K));
  HBPC_RUN(x, HBPC_PHASE_DOT, 1, k_cgs_update_dot<S><<<x->nblocks, kVecThreads, m1 * (kVecWarps + 1) * sizeof(double), x->stream>>>(K));
  HBPC_RUN(x, HBPC_PHASE_UPDATE, 1, k_cgs_update<S><<<x->nblocks, kVecThreads, m1 * sizeof(double), x->stream>>>(K));
  HBPC_RUN(x, HBPC_PHASE_UPDATE, 1, k_cgs_finalize<S><<<1, kVecThreads, 3 * (m1 + 1) * sizeof(double), x->stream>>>(K));
}

// Batches: the GMRES system of a group is scaled row-wise per instance,
// D J dX = -D G with D_i = 1 / ||G_i|| (0 for converged instances), so that
// its global relative tolerance asks the same relative accuracy of every
// instance (J is block diagonal over instances: dX is unchanged).  Applied to
// G before GMRES and to every Jacobian-vector product.
template <typename T>
hbpc_status inst_scale(hbpc_ctx* x, T* v, const int* col, int col_offset, const int* skip) {
  if (x->ninst == 0) return HBPC_OK;
  const dim3 grid(64, x->ninst);
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1,
           k_inst_scale<T><<<grid, 256, 0, x->stream>>>(v, size_t(x->ndof), x->d_irange, x->d_iscale, col,
                                                       col_offset, size_t(2 * x->ndof), skip));
  HBPC_LAUNCH_CK(x, "k_inst_scale");
  return HBPC_OK;
}

// Columns orthogonalised against by the Arnoldi iterations that took the
// cycle from column j0 to j1: sum_{j = j0}^{j1 - 1} (j + 1).
long long arnoldi_cols(int j0, int j1) {
  if (j1 <= j0) return 0;
  return (long long)(j1 - j0) * (j0 + j1 + 1) / 2;
}

hbpc_status arnoldi_step(hbpc_ctx* x) {
  hbpc_status s;
  if (x->sol.pc != HBPC_PC_NONE) {
    s = pc_apply(x, x->V, &x->st->j, x->K.vscale, x->Z, 0, &x->st->done);
    if (s != HBPC_OK) return s;
  }
  s = apply_jv(x, krylov_input(x));
  if (s != HBPC_OK) return s;
  if ((s = inst_scale<double>(x, x->V, &x->st->j, 1, &x->st->done)) != HBPC_OK) return s;
  cgs_launch<double>(x, x->K);
  HBPC_LAUNCH_CK(x, "arnoldi");
  return HBPC_OK;
}

hbpc_status arnoldi_step_f(hbpc_ctx* x);
hbpc_status arnoldi_step_schur(hbpc_ctx* x);

// One batch of Arnoldi steps.  Every launch of a step takes its column index,
// scale and stopping flag from device memory, so a batch is the same launch
// sequence every time: it is captured into a CUDA graph once per context (again
// when a launch shape changes) and replayed with one cudaGraphLaunch.  Direct
// launches instead with HBPC_GRAPH=0, during a phase-profiled step (its events
// would be captured), when the caller is capturing the stream, and after the
// runtime refused a capture (e.g. of the cooperative launch).
// kind 0: FP64 extended system, 1: mixed (FP32 Krylov loop), 2: FP64 Schur form
hbpc_status arnoldi_batch(hbpc_ctx* x, int batch, int kind) {
  hbpc_status (*step)(hbpc_ctx*) = kind == 1 ? arnoldi_step_f : kind == 2 ? arnoldi_step_schur : arnoldi_step;
  auto& g = x->arn_graph[kind];
  bool use = x->graph_mode != 0 && !x->prof.on && !g.failed;
  if (use) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(x->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) use = false;
  }
  if (use) {
    const long long key[8] = {x->nblocks, x->pc_threads, x->pc_grid, (long long)x->pc_smem, x->pc_shared ? 1 : 0,
                              x->coop ? 1 : 0, x->sol.pc, batch};
    if (g.exec && std::memcmp(key, g.key, sizeof(key)) != 0) {
      cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
    }
    if (!g.exec) {
      const long long l0 = x->stats.launches;
      const std::string err0 = x->err;
      cudaGraph_t graph = nullptr;
      bool ok = cudaStreamBeginCapture(x->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        hbpc_status s = HBPC_OK;
        for (int b = 0; b < batch && s == HBPC_OK; ++b) s = step(x);
        const cudaError_t e = cudaStreamEndCapture(x->stream, &graph);
        ok = s == HBPC_OK && e == cudaSuccess && graph != nullptr;
      }
      if (ok) ok = cudaGraphInstantiate(&g.exec, graph, 0) == cudaSuccess;
      if (graph) cudaGraphDestroy(graph);
      g.launches = x->stats.launches - l0;
      x->stats.launches = l0;   // the capture ran nothing
      if (!ok) {
        g.exec = nullptr;
        g.failed = true;
        (void)cudaGetLastError();   // the refused capture's error is not the caller's
        x->err = err0;
        if (x->verbose) std::fprintf(stderr, "[hbpc] Arnoldi batch not captured: direct launches\n");
      } else {
        std::memcpy(g.key, key, sizeof(key));
      }
    }
    if (g.exec) {
      HBPC_CK(x, cudaGraphLaunch(g.exec, x->stream));
      x->stats.launches += g.launches;
      return HBPC_OK;
    }
  }
  for (int b = 0; b < batch; ++b) {
    const hbpc_status s = step(x);
    if (s != HBPC_OK) return s;
  }
  return HBPC_OK;
}

// A restarted GMRES solve of J dX = -G (G in x->G with squared norms in
// st->nrm) from dX = 0, split into the pieces that the host-driven loop
// (gmres_run) and the device-driven step graph both launch:
//   init     dX = 0, V_0 = -G, the first cycle's state;
//   columns  a batch of Arnoldi columns (their kernels skip once the cycle's
//            done flag is set);
//   finish   end of a cycle: the small solve and dX += P^-1 V y;
//   restart  V_0 = -G - J dX and the next cycle's state.
// Kinds: the FP64 Krylov loop, the mixed (FP32) one, and the per-instance
// FP32 GMRES of a batch group (batch_krylov.cuh).
enum GmresKind { GM_FP64 = 0, GM_MIXED = 1, GM_BATCH = 2 };
constexpr int kGmresBatch = 4;   // Arnoldi columns between two looks at the state

hbpc_status gmres_init_fp64(hbpc_ctx* x) {
  const size_t n2 = size_t(2 * x->ndof);
  HBPC_CK(x, cudaMemsetAsync(x->dX, 0, n2 * sizeof(double), x->stream));
  HBPC_CK(x, cudaMemcpyAsync(x->V, x->G, n2 * sizeof(double), cudaMemcpyDeviceToDevice, x->stream));
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_cycle_init<double><<<1, 32, 0, x->stream>>>(x->K, -1.0, x->sol.tol_gmres_rel, 1, x->sol.gmres_max_iter));
  HBPC_LAUNCH_CK(x, "k_cycle_init");
  return HBPC_OK;
}

hbpc_status gmres_finish_fp64(hbpc_ctx* x) {
  hbpc_status s;
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_solve_y<double><<<1, 32, 0, x->stream>>>(x->K));
  if (x->sol.pc != HBPC_PC_NONE) {   // dX += P^-1 (V y)
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_combine<double, double><<<x->nblocks, kVecThreads, sizeof(double) * size_t(x->K.m + 1), x->stream>>>(x->K, x->Z, 0));
    s = pc_apply(x, x->Z, nullptr, nullptr, x->dX, 1, nullptr);
    if (s != HBPC_OK) return s;
  } else {
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_combine<double, double><<<x->nblocks, kVecThreads, sizeof(double) * size_t(x->K.m + 1), x->stream>>>(x->K, x->dX, 1));
  }
  HBPC_LAUNCH_CK(x, "gmres update");
  return HBPC_OK;
}

hbpc_status gmres_restart_fp64(hbpc_ctx* x) {
  const size_t n2 = size_t(2 * x->ndof);
  hbpc_status s = norms(x, x->dX, n2, x->dxn);
  if (s != HBPC_OK) return s;
  JvInput z{};
  z.V = x->dX; z.ld = n2; z.half = size_t(x->ndof);
  z.jidx = nullptr; z.vscale = nullptr;
  z.nrmW = x->dxn + 1; z.nrmS = x->dxn + 2;
  z.skip = nullptr;
  z.out = x->V + n2; z.out_ld = n2; z.out_offset = 0; z.out_jidx = nullptr;
  s = apply_jv(x, z);
  if (s != HBPC_OK) return s;
  if ((s = inst_scale<double>(x, x->V + n2, nullptr, 0, nullptr)) != HBPC_OK) return s;
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_neg_sum<<<grid_for(n2), 256, 0, x->stream>>>(x->G, x->V + n2, x->V, n2));
  s = norms(x, x->V, n2);
  if (s != HBPC_OK) return s;
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_cycle_init<double><<<1, 32, 0, x->stream>>>(x->K, 1.0, x->sol.tol_gmres_rel, 0, x->sol.gmres_max_iter));
  HBPC_LAUNCH_CK(x, "k_cycle_init");
  return HBPC_OK;
}

hbpc_status gmres_init(hbpc_ctx* x, int kind);
hbpc_status gmres_columns(hbpc_ctx* x, int kind);
hbpc_status gmres_finish(hbpc_ctx* x, int kind);
hbpc_status gmres_restart(hbpc_ctx* x, int kind);

// The host-driven loop: a look at the GMRES state after every batch of
// columns; *its / *conv as the solve ended (a solve that reaches its
// iteration cap returns with *conv false, Newton goes on).
hbpc_status gmres_run(hbpc_ctx* x, int kind, int* its_out, bool* conv_out) {
  hbpc_status s;
  if ((s = gmres_init(x, kind)) != HBPC_OK) return s;
  int j_prev = 0;
  for (;;) {
    if ((s = gmres_columns(x, kind)) != HBPC_OK) return s;
    if ((s = read_state(x)) != HBPC_OK) return s;
    const GmresState& h = *x->st_host;
    x->stats.arnoldi_cols += arnoldi_cols(j_prev, h.j);
    j_prev = h.j;
    if (kind != GM_BATCH && (!(h.resid == h.resid) || std::isinf(h.resid)))
      return fail(x, HBPC_ERR_NONFINITE, "GMRES residual is not finite");
    if (!h.done) continue;
    if ((s = gmres_finish(x, kind)) != HBPC_OK) return s;
    if (h.converged || h.its >= h.max_its) {
      *its_out = h.its;
      *conv_out = h.converged != 0;
      return HBPC_OK;
    }
    if ((s = gmres_restart(x, kind)) != HBPC_OK) return s;
    j_prev = 0;
  }
}

hbpc_status gmres(hbpc_ctx* x, int* its_out, bool* conv_out) { return gmres_run(x, GM_FP64, its_out, conv_out); }

// ---------------------------------------------------------------------------
// Mixed precision: the Krylov loop in FP32 (basis, Jacobian-vector product
// with the analytic linearised operator, BJ_ext apply), the Newton residual,
// update and stage logic in FP64.  Hessenberg, Givens rotations and the
// cross-thread / cross-block sums of the Arnoldi reductions stay FP64.
// ---------------------------------------------------------------------------
// ---- Schur form of the Newton system (Sec. 3.2.4, Eq. 19) -----------------
// The Krylov vectors are 2 n vectors whose sigma half is zero, so the basis,
// the Arnoldi column, the small solve and the combination are those of the
// extended system; only the product and the right-hand side differ.

// The extended product (Eq. 23/24) at X on the 2 n vector `in` into `out`
// (norms of in's halves first when the difference quotients need them).
hbpc_status jv_plain(hbpc_ctx* x, const double* in, double* out, const int* skip) {
  const size_t n2 = size_t(2 * x->ndof);
  if (!x->ops.jv_linear) {
    hbpc_status s = norms(x, in, n2, x->snrm);
    if (s != HBPC_OK) return s;
  }
  JvInput z{};
  z.V = in; z.ld = n2; z.half = size_t(x->ndof);
  z.nrmW = x->snrm + 1; z.nrmS = x->snrm + 2;
  z.skip = skip;
  z.out = out; z.out_ld = n2; z.out_offset = 0;
  return apply_jv(x, z);
}

// J_Schur z = the first half of the extended product on (z, dR1/dW z): sa
// holds (z, 0) on entry, (z, J z) on exit; the product goes to `out`
// (column *out_jidx + out_offset of out when out_jidx is given).
hbpc_status schur_product(hbpc_ctx* x, double* out, const int* out_jidx, int out_offset, const int* skip) {
  const size_t n = size_t(x->ndof), n2 = 2 * n;
  hbpc_status s = jv_plain(x, x->sa, x->sb, skip);              // sb = (.., -J z)
  if (s != HBPC_OK) return s;
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_schur_pair<<<grid_for(n), 256, 0, x->stream>>>(x->sa, x->sb, n, skip));
  if (!x->ops.jv_linear && (s = norms(x, x->sa, n2, x->snrm)) != HBPC_OK) return s;
  JvInput z{};
  z.V = x->sa; z.ld = n2; z.half = n;
  z.nrmW = x->snrm + 1; z.nrmS = x->snrm + 2;
  z.skip = skip;
  z.out = out; z.out_ld = n2; z.out_offset = out_offset; z.out_jidx = out_jidx;
  if ((s = apply_jv(x, z)) != HBPC_OK) return s;
  HBPC_LAUNCH_CK(x, "Schur product");
  return HBPC_OK;
}

// One Arnoldi iteration of the Schur system: z = P^-1 v_j (the D block of
// BJ_ext: its apply on (v_j, 0) has M v_j in the first half), the product
// J_Schur z into column j + 1 (its sigma half cleared), the CGS column.
hbpc_status arnoldi_step_schur(hbpc_ctx* x) {
  const size_t n = size_t(x->ndof), n2 = 2 * n;
  const int* jd = &x->st->j;
  const int* skip = &x->st->done;
  hbpc_status s;
  if (x->sol.pc != HBPC_PC_NONE) {
    if ((s = pc_apply(x, x->V, jd, x->K.vscale, x->sa, 0, skip)) != HBPC_OK) return s;
    HBPC_RUN(x, HBPC_PHASE_PC, 1, k_zero_half<<<grid_for(n), 256, 0, x->stream>>>(x->sa, nullptr, 0, n, skip));
  } else {
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1,
             k_gather_col<<<grid_for(n2), 256, 0, x->stream>>>(x->V, jd, x->K.vscale, x->sa, n2, skip));
  }
  if ((s = schur_product(x, x->V, jd, 1, skip)) != HBPC_OK) return s;
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_zero_half<<<grid_for(n), 256, 0, x->stream>>>(x->V, jd, 1, n, skip));
  cgs_launch<double>(x, x->K);
  HBPC_LAUNCH_CK(x, "arnoldi (Schur)");
  return HBPC_OK;
}

// GMRES on J_Schur dW = -G1 + c2 (dR2/dsigma) G2 (right preconditioned by the
// BJ_ext D blocks when there is a preconditioner); dW into the first half of
// x->dX.  G = (G1, G2) is the current residual.
hbpc_status gmres_schur(hbpc_ctx* x, int* its_out, bool* conv_out) {
  const size_t n = size_t(x->ndof), n2 = 2 * n;
  HBPC_CK(x, cudaMemsetAsync(x->dX, 0, n2 * sizeof(double), x->stream));
  // right-hand side: the extended product on (G2, 0) has -J G2 in its second half
  HBPC_CK(x, cudaMemcpyAsync(x->sa, x->G + n, n * sizeof(double), cudaMemcpyDeviceToDevice, x->stream));
  HBPC_CK(x, cudaMemsetAsync(x->sa + n, 0, n * sizeof(double), x->stream));
  hbpc_status s = jv_plain(x, x->sa, x->sb, nullptr);
  if (s != HBPC_OK) return s;
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_schur_rhs<<<grid_for(n), 256, 0, x->stream>>>(x->G, x->sb, x->c12, x->srhs, n));
  HBPC_CK(x, cudaMemcpyAsync(x->V, x->srhs, n2 * sizeof(double), cudaMemcpyDeviceToDevice, x->stream));
  if ((s = norms(x, x->V, n2)) != HBPC_OK) return s;
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_cycle_init<double><<<1, 32, 0, x->stream>>>(x->K, 1.0, x->sol.tol_gmres_rel, 1, x->sol.gmres_max_iter));
  HBPC_LAUNCH_CK(x, "k_cycle_init (Schur)");
  const int batch = 4;
  int j_prev = 0;
  for (;;) {
    if ((s = arnoldi_batch(x, batch, 2)) != HBPC_OK) return s;
    if ((s = read_state(x)) != HBPC_OK) return s;
    const GmresState& h = *x->st_host;
    x->stats.arnoldi_cols += arnoldi_cols(j_prev, h.j);
    j_prev = h.j;
    if (!(h.resid == h.resid) || std::isinf(h.resid))
      return fail(x, HBPC_ERR_NONFINITE, "GMRES residual is not finite (Schur)");
    if (!h.done) continue;
    // end of a cycle: dW += P^-1 V y
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_solve_y<double><<<1, 32, 0, x->stream>>>(x->K));
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_combine<double, double><<<x->nblocks, kVecThreads, sizeof(double) * size_t(x->K.m + 1), x->stream>>>(x->K, x->sa, 0));
    if (x->sol.pc != HBPC_PC_NONE) {
      if ((s = pc_apply(x, x->sa, nullptr, nullptr, x->sb, 0, nullptr)) != HBPC_OK) return s;
      HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_add_half<<<grid_for(n), 256, 0, x->stream>>>(x->sb, x->dX, n));
    } else {
      HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_add_half<<<grid_for(n), 256, 0, x->stream>>>(x->sa, x->dX, n));
    }
    HBPC_LAUNCH_CK(x, "GMRES update (Schur)");
    if (h.converged || h.its >= h.max_its) {
      *its_out = h.its;
      *conv_out = h.converged != 0;
      return HBPC_OK;
    }
    // restart: V_0 = rhs - J_Schur dW
    HBPC_CK(x, cudaMemcpyAsync(x->sa, x->dX, n * sizeof(double), cudaMemcpyDeviceToDevice, x->stream));
    HBPC_CK(x, cudaMemsetAsync(x->sa + n, 0, n * sizeof(double), x->stream));
    if ((s = schur_product(x, x->sb, nullptr, 0, nullptr)) != HBPC_OK) return s;
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_schur_restart<<<grid_for(n), 256, 0, x->stream>>>(x->srhs, x->sb, x->V, n));
    if ((s = norms(x, x->V, n2)) != HBPC_OK) return s;
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_cycle_init<double><<<1, 32, 0, x->stream>>>(x->K, 1.0, x->sol.tol_gmres_rel, 0, x->sol.gmres_max_iter));
    HBPC_LAUNCH_CK(x, "k_cycle_init (Schur restart)");
    j_prev = 0;
  }
}

// sigma increment of the Schur form: dX_S = -G2 + (dR1/dW) dW
hbpc_status schur_sigma(hbpc_ctx* x) {
  const size_t n = size_t(x->ndof);
  HBPC_CK(x, cudaMemcpyAsync(x->sa, x->dX, n * sizeof(double), cudaMemcpyDeviceToDevice, x->stream));
  HBPC_CK(x, cudaMemsetAsync(x->sa + n, 0, n * sizeof(double), x->stream));
  hbpc_status s = jv_plain(x, x->sa, x->sb, nullptr);
  if (s != HBPC_OK) return s;
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_schur_sigma<<<grid_for(n), 256, 0, x->stream>>>(x->G, x->sb, x->dX, n));
  HBPC_LAUNCH_CK(x, "Schur sigma");
  return HBPC_OK;
}

JvInputT<float> krylov_input_f(hbpc_ctx* x) {
  JvInputT<float> z{};
  z.V = x->Vf; z.ld = size_t(2 * x->ndof); z.half = size_t(x->ndof);
  z.jidx = &x->st->j;
  z.vscale = x->Kf.vscale;
  z.nrmW = x->Kf.nrmW; z.nrmS = x->Kf.nrmS;
  z.skip = &x->st->done;
  z.out = x->Vf; z.out_ld = size_t(2 * x->ndof); z.out_offset = 1;
  z.out_jidx = &x->st->j;
  if (x->sol.pc != HBPC_PC_NONE) {
    z.V = x->Zf; z.jidx = nullptr; z.vscale = nullptr;
    z.nrmW = x->zn + 1; z.nrmS = x->zn + 2;
  }
  return z;
}

hbpc_status apply_jv_f(hbpc_ctx* x, const JvInputT<float>& z) {
  HBPC_RUN(x, HBPC_PHASE_JV, 1,
           x->ops.jv_f(x->prmf, z, jv_coef(x), x->Wf, x->Wf + x->ndof, x->stream));
  HBPC_LAUNCH_CK(x, "jv_f");
  return HBPC_OK;
}

hbpc_status arnoldi_step_f(hbpc_ctx* x) {
  hbpc_status s;
  if (x->sol.pc != HBPC_PC_NONE) {
    s = pc_apply_f(x, x->Vf, &x->st->j, x->Kf.vscale, x->Zf, 0, &x->st->done);
    if (s != HBPC_OK) return s;
  }
  if ((s = apply_jv_f(x, krylov_input_f(x))) != HBPC_OK) return s;
  if ((s = inst_scale<float>(x, x->Vf, &x->st->j, 1, &x->st->done)) != HBPC_OK) return s;
  cgs_launch<float>(x, x->Kf);
  HBPC_LAUNCH_CK(x, "arnoldi<float>");
  return HBPC_OK;
}

hbpc_status gmres_init_mixed(hbpc_ctx* x) {
  const size_t n2 = size_t(2 * x->ndof);
  hbpc_status s;
  HBPC_CK(x, cudaMemsetAsync(x->dX, 0, n2 * sizeof(double), x->stream));
  if ((s = to_float(x, x->G, x->Vf, n2)) != HBPC_OK) return s;
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_cycle_init<float><<<1, 32, 0, x->stream>>>(x->Kf, -1.0, x->sol.tol_gmres_rel, 1, x->sol.gmres_max_iter));
  HBPC_LAUNCH_CK(x, "k_cycle_init<float>");
  return HBPC_OK;
}

hbpc_status gmres_finish_mixed(hbpc_ctx* x) {
  const size_t n2 = size_t(2 * x->ndof);
  hbpc_status s;
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_solve_y<float><<<1, 32, 0, x->stream>>>(x->Kf));
  const size_t smy = sizeof(double) * size_t(x->Kf.m + 1);
  if (x->sol.pc != HBPC_PC_NONE) {   // dX += P^-1 (V y)
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_combine<float, float><<<x->nblocks, kVecThreads, smy, x->stream>>>(x->Kf, x->Zf, 0));
    if ((s = pc_apply_f(x, x->Zf, nullptr, nullptr, x->Zf2, 0, nullptr)) != HBPC_OK) return s;
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_add_float<<<grid_for(n2), 256, 0, x->stream>>>(x->Zf2, x->dX, n2));
  } else {
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_combine<float, double><<<x->nblocks, kVecThreads, smy, x->stream>>>(x->Kf, x->dX, 1));
  }
  HBPC_LAUNCH_CK(x, "gmres<float> update");
  return HBPC_OK;
}

// restart: V_0 = -G - J dX (FP32 Jacobian-vector product of the FP32 copy of dX)
hbpc_status gmres_restart_mixed(hbpc_ctx* x) {
  const size_t n2 = size_t(2 * x->ndof);
  hbpc_status s;
  if ((s = to_float(x, x->dX, x->Zf, n2)) != HBPC_OK) return s;
  JvInputT<float> z{};
  z.V = x->Zf; z.ld = n2; z.half = size_t(x->ndof);
  z.nrmW = x->zn + 1; z.nrmS = x->zn + 2;
  z.out = x->Vf + n2; z.out_ld = n2; z.out_offset = 0;
  if ((s = apply_jv_f(x, z)) != HBPC_OK) return s;
  if ((s = inst_scale<float>(x, x->Vf + n2, nullptr, 0, nullptr)) != HBPC_OK) return s;
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_neg_sum_f<<<grid_for(n2), 256, 0, x->stream>>>(x->G, x->Vf + n2, x->Vf, n2));
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_norms<double, float><<<x->nblocks, kVecThreads, 0, x->stream>>>(x->Vf, n2, size_t(x->ndof), x->K, nullptr));
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_cycle_init<float><<<1, 32, 0, x->stream>>>(x->Kf, 1.0, x->sol.tol_gmres_rel, 0, x->sol.gmres_max_iter));
  HBPC_LAUNCH_CK(x, "gmres<float> restart");
  return HBPC_OK;
}

hbpc_status gmres_f(hbpc_ctx* x, int* its_out, bool* conv_out) { return gmres_run(x, GM_MIXED, its_out, conv_out); }

// Per-instance GMRES of a batch group in the mixed mode: J dX = -G for every
// active instance with its own Krylov space (batch_krylov.cuh); converged
// instances (zero right-hand side after the Newton freeze) take no step.
hbpc_status gmres_bstart(hbpc_ctx* x, double sign, int first) {
  BKrylovT<float>& K = x->BK;
  const int grid = x->bk_grid;
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_btile_sqnorm<float><<<grid, kVecThreads, 0, x->stream>>>(K));
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_bcycle_init<float><<<1, 256, 0, x->stream>>>(K, sign, x->sol.tol_gmres_rel, first, x->sol.gmres_max_iter));
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_bscale0<float><<<grid, kVecThreads, 0, x->stream>>>(K));
  HBPC_LAUNCH_CK(x, "batched cycle start");
  return HBPC_OK;
}

hbpc_status gmres_init_batch(hbpc_ctx* x) {
  const size_t n2 = size_t(2 * x->ndof);
  hbpc_status s;
  HBPC_CK(x, cudaMemsetAsync(x->dX, 0, n2 * sizeof(double), x->stream));
  if ((s = to_float(x, x->G, x->Vf, n2)) != HBPC_OK) return s;
  return gmres_bstart(x, -1.0, 1);
}

hbpc_status gmres_columns_batch(hbpc_ctx* x) {
  const size_t n2 = size_t(2 * x->ndof);
  BKrylovT<float>& K = x->BK;
  const size_t shm = size_t(K.m + 1) * (kVecWarps + 1) * sizeof(double);
  hbpc_status s;
  for (int b = 0; b < kGmresBatch; ++b) {
    if (x->sol.pc != HBPC_PC_NONE &&
        (s = pc_apply_f(x, x->Vf, &x->st->j, nullptr, x->Zf, 0, &x->st->done)) != HBPC_OK)
      return s;
    JvInputT<float> z{};
    z.V = x->sol.pc != HBPC_PC_NONE ? x->Zf : x->Vf;
    z.ld = n2; z.half = size_t(x->ndof);
    z.jidx = x->sol.pc != HBPC_PC_NONE ? nullptr : &x->st->j;
    z.nrmW = x->zn + 1; z.nrmS = x->zn + 2;   // not read by the FP32 products
    z.skip = &x->st->done;
    z.out = x->Vf; z.out_ld = n2; z.out_offset = 1; z.out_jidx = &x->st->j;
    if ((s = apply_jv_f(x, z)) != HBPC_OK) return s;
    void* args[] = {&K};
    HBPC_RUN(x, HBPC_PHASE_DOT, 1,
             cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_bcgs_coop<float>), dim3(x->bk_grid),
                                         dim3(kVecThreads), args, shm, x->stream));
    HBPC_LAUNCH_CK(x, "k_bcgs_coop");
  }
  return HBPC_OK;
}

hbpc_status gmres_finish_batch(hbpc_ctx* x) {
  const size_t n2 = size_t(2 * x->ndof);
  BKrylovT<float>& K = x->BK;
  const int grid = x->bk_grid;
  hbpc_status s;
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_bsolve_y<float><<<(K.ninst + 7) / 8, 256, 0, x->stream>>>(K));
  if (x->sol.pc != HBPC_PC_NONE) {   // dX += P^-1 (V y)
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_bcombine<float, float><<<grid, kVecThreads, 0, x->stream>>>(K, x->Zf, 0));
    if ((s = pc_apply_f(x, x->Zf, nullptr, nullptr, x->Zf2, 0, nullptr)) != HBPC_OK) return s;
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_add_float<<<grid_for(n2), 256, 0, x->stream>>>(x->Zf2, x->dX, n2));
  } else {
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_bcombine<float, double><<<grid, kVecThreads, 0, x->stream>>>(K, x->dX, 1));
  }
  HBPC_LAUNCH_CK(x, "batched gmres update");
  return HBPC_OK;
}

// restart: V_0 = -G - J dX, every instance from its own residual
hbpc_status gmres_restart_batch(hbpc_ctx* x) {
  const size_t n2 = size_t(2 * x->ndof);
  hbpc_status s;
  if ((s = to_float(x, x->dX, x->Zf, n2)) != HBPC_OK) return s;
  JvInputT<float> z{};
  z.V = x->Zf; z.ld = n2; z.half = size_t(x->ndof);
  z.nrmW = x->zn + 1; z.nrmS = x->zn + 2;
  z.out = x->Vf + n2; z.out_ld = n2; z.out_offset = 0;
  if ((s = apply_jv_f(x, z)) != HBPC_OK) return s;
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_neg_sum_f<<<grid_for(n2), 256, 0, x->stream>>>(x->G, x->Vf + n2, x->Vf, n2));
  return gmres_bstart(x, 1.0, 0);
}

hbpc_status gmres_bf(hbpc_ctx* x, int* its_out, bool* conv_out) { return gmres_run(x, GM_BATCH, its_out, conv_out); }

hbpc_status gmres_init(hbpc_ctx* x, int kind) {
  return kind == GM_FP64 ? gmres_init_fp64(x) : kind == GM_MIXED ? gmres_init_mixed(x) : gmres_init_batch(x);
}
hbpc_status gmres_columns(hbpc_ctx* x, int kind) {
  return kind == GM_BATCH ? gmres_columns_batch(x) : arnoldi_batch(x, kGmresBatch, kind);
}
hbpc_status gmres_finish(hbpc_ctx* x, int kind) {
  return kind == GM_FP64 ? gmres_finish_fp64(x) : kind == GM_MIXED ? gmres_finish_mixed(x) : gmres_finish_batch(x);
}
hbpc_status gmres_restart(hbpc_ctx* x, int kind) {
  return kind == GM_FP64 ? gmres_restart_fp64(x) : kind == GM_MIXED ? gmres_restart_mixed(x) : gmres_restart_batch(x);
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
hbpc_status newton_batch(hbpc_ctx* x, const double* b, double a1, double a2, const double* W0);

hbpc_status newton(hbpc_ctx* x, const double* b, double a1, double a2, const double* W0) {
  if (x->ninst > 0) return newton_batch(x, b, a1, a2, W0);
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
  if (!std::isfinite(g0)) return nonfinite(x, "initial Newton residual is not finite");
  x->stats.newton_solves += 1;
  if (x->verbose) std::fprintf(stderr, "[hbpc] newton a1=%g a2=%g ||G0||=%.6e\n", a1, a2, g0);
  if (g0 == 0.0) return HBPC_OK;
  for (int r = 0; r < x->sol.newton_max_iter; ++r) {
    int its = 0;
    bool conv = false;
    if (x->sol.pc != HBPC_PC_NONE && (x->pc_every || r == 0) && (s = pc_build(x, x->X, c1, c2)) != HBPC_OK) return s;
    if (x->schur) {
      if ((s = gmres_schur(x, &its, &conv)) != HBPC_OK) return s;
      if ((s = schur_sigma(x)) != HBPC_OK) return s;
    } else if (x->sol.precision == HBPC_PREC_MIXED) {
      if ((s = to_float(x, x->X, x->Wf, size_t(2 * n))) != HBPC_OK) return s;
      if ((s = gmres_f(x, &its, &conv)) != HBPC_OK) return s;
    } else {
      if ((s = gmres(x, &its, &conv)) != HBPC_OK) return s;
    }
    x->stats.gmres_its += its;
    x->stats.newton_its += 1;
    const int per = (x->ops.jv_linear ? 2 : 3) * (x->schur ? 2 : 1);
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
      return nonfinite(x, "Newton residual is not finite");
    if (gn <= x->sol.tol_newton_rel * g0 || dW <= x->sol.tol_newton_abs) return HBPC_OK;
  }
  return fail(x, HBPC_ERR_NO_CONVERGENCE, "Newton did not converge within newton_max_iter");
}

// Per-instance squared norms of a 2 n_dof vector into x->h_inrm.
hbpc_status inst_norms(hbpc_ctx* x, const double* v) {
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1,
           k_inst_sqnorms<<<x->ninst, kInstThreads, 0, x->stream>>>(v, size_t(x->ndof), x->d_irange, x->d_inrm));
  HBPC_LAUNCH_CK(x, "k_inst_sqnorms");
  HBPC_CK(x, cudaMemcpyAsync(x->h_inrm.data(), x->d_inrm, 2 * x->ninst * sizeof(double), cudaMemcpyDeviceToHost,
                             x->stream));
  return sync(x, "instance norms");
}

// Newton for a batch of independent instances: one extended system, one GMRES
// per Newton iteration over all still-active instances (the Jacobian and the
// block preconditioner are block diagonal over instances, so a zero
// right-hand side keeps an instance's update exactly zero), and the stopping
// tests of Sec. 3.2.1 applied to every instance separately: ||G_i|| <=
// tol ||G_i^0|| or ||dW_i|| <= tol_abs.  A converged instance is frozen.
hbpc_status newton_batch(hbpc_ctx* x, const double* b, double a1, double a2, const double* W0) {
  const long long n = x->ndof;
  const int ni = x->ninst;
  const double dt = x->sol.dt;
  const double c1 = a1 * dt, c2 = a2 * dt * dt / 2.0;
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_set2<<<1, 32, 0, x->stream>>>(x->c12, c1, c2));
  if (W0 != x->X) HBPC_CK(x, cudaMemcpyAsync(x->X, W0, n * sizeof(double), cudaMemcpyDeviceToDevice, x->stream));
  HBPC_RUN(x, HBPC_PHASE_OPERATOR, 1, x->ops.r1(x->prm, x->X, x->X + n, x->stream));
  HBPC_LAUNCH_CK(x, "r1");
  x->stats.r1_evals += 1;
  hbpc_status s = residual(x, b, c1, c2);
  if (s != HBPC_OK) return s;
  if ((s = inst_norms(x, x->G)) != HBPC_OK) return s;
  std::vector<double> g0(ni);
  int nact = 0;
  for (int i = 0; i < ni; ++i) {
    g0[i] = std::sqrt(x->h_inrm[2 * i]);
    if (!std::isfinite(g0[i])) return fail(x, HBPC_ERR_NONFINITE, "initial Newton residual is not finite");
    x->h_active[i] = g0[i] > 0.0 ? 1 : 0;
    nact += x->h_active[i];
  }
  x->stats.newton_solves += 1;
  for (int r = 0; nact > 0; ++r) {
    if (r >= x->sol.newton_max_iter)
      return fail(x, HBPC_ERR_NO_CONVERGENCE, "Newton did not converge within newton_max_iter (batch)");
    // per-instance GMRES (x->bk): active instances as they are, converged ones
    // with a zero right-hand side; the shared GMRES: rows scaled by 1 / ||G_i||
    for (int i = 0; i < ni; ++i)
      x->h_iscale[i] = !x->h_active[i] ? 0.0 : x->bk ? 1.0 : 1.0 / std::sqrt(x->h_inrm[2 * i]);
    HBPC_CK(x, cudaMemcpyAsync(x->d_iscale, x->h_iscale.data(), ni * sizeof(double), cudaMemcpyHostToDevice,
                               x->stream));
    if ((s = inst_scale<double>(x, x->G, nullptr, 0, nullptr)) != HBPC_OK) return s;
    if ((s = norms(x, x->G, size_t(2 * n))) != HBPC_OK) return s;   // of the scaled right-hand side
    int its = 0;
    bool conv = false;
    if (x->sol.pc != HBPC_PC_NONE && (x->pc_every || r == 0) && (s = pc_build(x, x->X, c1, c2)) != HBPC_OK) return s;
    if (x->sol.precision == HBPC_PREC_MIXED) {
      if ((s = to_float(x, x->X, x->Wf, size_t(2 * n))) != HBPC_OK) return s;
      if ((s = (x->bk ? gmres_bf(x, &its, &conv) : gmres_f(x, &its, &conv))) != HBPC_OK) return s;
    } else {
      if ((s = gmres(x, &its, &conv)) != HBPC_OK) return s;
    }
    x->stats.gmres_its += its;
    x->stats.newton_its += 1;
    const int per = x->ops.jv_linear ? 2 : 3;
    x->stats.r1_evals += (long long)its * (x->ops.jv_linear ? 2 : 1);
    x->stats.r2_evals += (long long)its * (per - (x->ops.jv_linear ? 2 : 1));
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_add<<<grid_for(size_t(2 * n)), 256, 0, x->stream>>>(x->dX, x->X, size_t(2 * n)));
    HBPC_LAUNCH_CK(x, "newton update");
    if ((s = inst_norms(x, x->dX)) != HBPC_OK) return s;
    std::vector<double> dW(ni);
    for (int i = 0; i < ni; ++i) dW[i] = std::sqrt(x->h_inrm[2 * i + 1]);
    if ((s = residual(x, b, c1, c2)) != HBPC_OK) return s;
    if ((s = inst_norms(x, x->G)) != HBPC_OK) return s;
    nact = 0;
    for (int i = 0; i < ni; ++i) {
      if (!x->h_active[i]) continue;
      const double gn = std::sqrt(x->h_inrm[2 * i]);
      if (!std::isfinite(gn) || !std::isfinite(dW[i]))
        return fail(x, HBPC_ERR_NONFINITE, "Newton residual is not finite (batch)");
      if (x->verbose)
        std::fprintf(stderr, "[hbpc] batch it %d inst %d gmres %d ||G||=%.6e rel %.3e ||dW||=%.3e\n", r, i, its, gn,
                     gn / g0[i], dW[i]);
      if (gn <= x->sol.tol_newton_rel * g0[i] || dW[i] <= x->sol.tol_newton_abs) x->h_active[i] = 0;
      nact += x->h_active[i];
    }
  }
  return HBPC_OK;
}

hbpc_status eval_r1r2(hbpc_ctx* x, const double* w, double* r1, double* r2) {
  HBPC_RUN(x, HBPC_PHASE_OPERATOR, 1, x->ops.r1(x->prm, w, r1, x->stream));
  HBPC_RUN(x, HBPC_PHASE_OPERATOR, 1, x->ops.r2(x->prm, w, r1, r2, x->stream));
  HBPC_LAUNCH_CK(x, "stage r1/r2");
  x->stats.r1_evals += 1;
  x->stats.r2_evals += 1;
  return HBPC_OK;
}

// One HBPC(q, k_max) step of Algorithm 1 on x->Wn, every implicit stage
// solved by `solve` (the host-driven Newton, or its graph form while the step
// is captured: then the new state is copied to x->Wn only if no solve failed,
// and nothing waits for the device).
using NewtonFn = hbpc_status (*)(hbpc_ctx*, const double*, double, double, const double*);
hbpc_status step_body(hbpc_ctx* x, NewtonFn solve, bool graph) {
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
    if ((st = solve(x, x->bvec, a1, a2, W(0, l - 1))) != HBPC_OK) return st;
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
    // right-hand side of corrector stage l (Eq. 6 with the quadrature I_l)
    auto rhs = [&](int l, double* out) -> hbpc_status {
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
      HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_lincomb<<<grid_for(size_t(n)), 256, 0, x->stream>>>(lc, out, size_t(n)));
      HBPC_LAUNCH_CK(x, "corrector rhs");
      return HBPC_OK;
    };
    if (x->cb && s > 1 && !graph) {
      // the s - 1 stages of this sweep depend only on level cur: one batched
      // Newton solve with stage l as instance l - 1 (Sec. 6 outlook)
      hbpc_ctx* g = x->cb;
      const size_t vpe = size_t(g->ndof / g->nE);
      for (int l = 1; l < s; ++l) {
        const size_t off = size_t(g->ie0[l - 1]) * vpe;
        if ((st = rhs(l, g->bvec + off)) != HBPC_OK) return st;
        HBPC_CK(x, cudaMemcpyAsync(g->stage + off, Wc(l), n * sizeof(double), cudaMemcpyDeviceToDevice, x->stream));
      }
      const hbpc_stats before = g->stats;
      st = newton(g, g->bvec, 1.0, 1.0, g->stage);
      x->stats.newton_solves += g->stats.newton_solves - before.newton_solves;
      x->stats.newton_its += g->stats.newton_its - before.newton_its;
      x->stats.gmres_its += g->stats.gmres_its - before.gmres_its;
      x->stats.r1_evals += g->stats.r1_evals - before.r1_evals;
      x->stats.r2_evals += g->stats.r2_evals - before.r2_evals;
      x->stats.launches += g->stats.launches - before.launches;
      x->stats.arnoldi_cols += g->stats.arnoldi_cols - before.arnoldi_cols;
      if (st != HBPC_OK) return fail(x, st, "corrector batch: " + g->err);
      for (int l = 1; l < s; ++l) {
        const size_t off = size_t(g->ie0[l - 1]) * vpe;
        HBPC_CK(x, cudaMemcpyAsync(W(nxt, l), g->X + off, n * sizeof(double), cudaMemcpyDeviceToDevice, x->stream));
        if ((st = eval_r1r2(x, W(nxt, l), R1(nxt, l), R2(nxt, l))) != HBPC_OK) return st;
      }
      cur = nxt;
      continue;
    }
    for (int l = 1; l < s; ++l) {
      if ((st = rhs(l, x->bvec)) != HBPC_OK) return st;
      if ((st = solve(x, x->bvec, 1.0, 1.0, Wc(l))) != HBPC_OK) return st;
      HBPC_CK(x, cudaMemcpyAsync(W(nxt, l), x->X, n * sizeof(double), cudaMemcpyDeviceToDevice, x->stream));
      if ((st = eval_r1r2(x, W(nxt, l), R1(nxt, l), R2(nxt, l))) != HBPC_OK) return st;
    }
    cur = nxt;
  }
  const double* last = (s - 1 == 0) ? W(0, 0) : W(cur, s - 1);
  if (graph) {
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_sg_copy_if_ok<<<grid_for(size_t(n)), 256, 0, x->stream>>>(last, x->Wn, size_t(n), x->sg.ctl));
    HBPC_LAUNCH_CK(x, "step result");
    return HBPC_OK;
  }
  HBPC_CK(x, cudaMemcpyAsync(x->Wn, last, n * sizeof(double), cudaMemcpyDeviceToDevice, x->stream));
  return sync(x, "hbpc step");
}

// ---- the step as one CUDA graph ----------------------------------------------
// The graph is captured segment by segment (cudaStreamBeginCaptureToGraph on a
// private stream): straight-line work between two loops is one captured
// segment, a loop or branch is a conditional node whose body graph is captured
// the same way.  Each level keeps its frontier (the nodes the next one depends
// on) and counts the kernels launched in it outside its nested bodies, which
// the control kernel of that level adds to the step's count every time it runs.
struct GBuild {
  hbpc_ctx* x;
  struct Level {
    cudaGraph_t g;
    std::vector<cudaGraphNode_t> front;
    long long l0, nested;
  };
  std::vector<Level> lv;
  cudaError_t e = cudaSuccess;
  bool open_seg = false;

  void begin() {
    if (e != cudaSuccess) return;
    Level& L = lv.back();
    e = cudaStreamBeginCaptureToGraph(x->stream, L.g, L.front.empty() ? nullptr : L.front.data(), nullptr,
                                      L.front.size(), cudaStreamCaptureModeThreadLocal);
    open_seg = e == cudaSuccess;
  }
  void end() {
    if (!open_seg) return;
    open_seg = false;
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaError_t e1 = cudaStreamGetCaptureInfo(x->stream, &cs, nullptr, nullptr, &deps, nullptr, &nd);
    std::vector<cudaGraphNode_t> f;
    if (e1 == cudaSuccess) f.assign(deps, deps + nd);
    cudaGraph_t out = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(x->stream, &out);
    if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2;
    if (e == cudaSuccess) lv.back().front = f;
  }
  cudaGraphConditionalHandle handle() {
    end();
    cudaGraphConditionalHandle h = 0;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, lv.back().g, 0, 0);
    begin();
    return h;
  }
  void open(cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type) {
    end();
    if (e != cudaSuccess) return;
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = type;
    p.conditional.size = 1;
    Level& L = lv.back();
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, L.g, L.front.empty() ? nullptr : L.front.data(), nullptr, L.front.size(), &p);
    if (e != cudaSuccess) return;
    L.front.assign(1, node);
    lv.push_back(Level{p.conditional.phGraph_out[0], {}, x->stats.launches, 0});
    begin();
  }
  void close() {
    end();
    const long long total = x->stats.launches - lv.back().l0;
    lv.pop_back();
    lv.back().nested += total;
    begin();
  }
  // kernels of the current level outside its nested bodies, plus one (the
  // control kernel about to be launched)
  int own() const { return int(x->stats.launches - lv.back().l0 - lv.back().nested) + 1; }
};

thread_local GBuild* g_build = nullptr;   // the builder of the step this thread captures

// The GMRES solve of gmres_run as nodes: a WHILE loop over batches of columns
// with the cycle end and the restart as nested IF branches.
hbpc_status gmres_graph(hbpc_ctx* x, GBuild& B, int kind) {
  hbpc_status s;
  if ((s = gmres_init(x, kind)) != HBPC_OK) return s;
  const cudaGraphConditionalHandle h_loop = B.handle();
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_sg_gmres_begin<<<1, 32, 0, x->stream>>>(x->sg.ctl, h_loop, 0));
  B.open(h_loop, cudaGraphCondTypeWhile);
  {
    const cudaGraphConditionalHandle h_end = B.handle();
    if ((s = gmres_columns(x, kind)) != HBPC_OK) return s;
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_sg_gmres_tick<<<1, 32, 0, x->stream>>>(x->st, x->sg.ctl, h_loop, h_end, kind != GM_BATCH ? 1 : 0, B.own()));
    B.open(h_end, cudaGraphCondTypeIf);
    {
      const cudaGraphConditionalHandle h_restart = B.handle();
      if ((s = gmres_finish(x, kind)) != HBPC_OK) return s;
      HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_sg_gmres_end<<<1, 32, 0, x->stream>>>(x->st, x->sg.ctl, h_loop, h_restart, B.own()));
      B.open(h_restart, cudaGraphCondTypeIf);
      if ((s = gmres_restart(x, kind)) != HBPC_OK) return s;
      HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_sg_count<<<1, 32, 0, x->stream>>>(x->sg.ctl, B.own()));
      B.close();
    }
    B.close();
  }
  B.close();
  HBPC_LAUNCH_CK(x, "gmres graph");
  return B.e == cudaSuccess ? HBPC_OK : cuda_fail(x, B.e, "gmres graph");
}

// Newton of `newton` / `newton_batch` as nodes: a WHILE loop whose control
// kernel applies the stopping tests; the evaluation counts of its body are
// taken out of the per-step (outside-the-loops) counts.
hbpc_status newton_graph(hbpc_ctx* x, const double* b, double a1, double a2, const double* W0) {
  GBuild& B = *g_build;
  const long long n = x->ndof;
  const size_t n2 = size_t(2 * n);
  const int ni = x->ninst;
  const double dt = x->sol.dt;
  const double c1 = a1 * dt, c2 = a2 * dt * dt / 2.0;
  hbpc_status s;
  HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_set2<<<1, 32, 0, x->stream>>>(x->c12, c1, c2));
  if (W0 != x->X) HBPC_CK(x, cudaMemcpyAsync(x->X, W0, n * sizeof(double), cudaMemcpyDeviceToDevice, x->stream));
  HBPC_RUN(x, HBPC_PHASE_OPERATOR, 1, x->ops.r1(x->prm, x->X, x->X + n, x->stream));
  HBPC_LAUNCH_CK(x, "r1");
  x->stats.r1_evals += 1;
  if ((s = residual(x, b, c1, c2)) != HBPC_OK) return s;
  auto inst_sq = [&](const double* v) {
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1,
             k_inst_sqnorms<<<ni, kInstThreads, 0, x->stream>>>(v, size_t(n), x->d_irange, x->d_inrm));
  };
  const int per_inst = x->bk ? 1 : 0;
  const cudaGraphConditionalHandle h_newton = B.handle();
  if (ni > 0) {
    inst_sq(x->G);
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_sg_newton_begin_batch<<<1, 256, 0, x->stream>>>(ni, x->d_inrm, x->sg.g0, x->sg.active, x->d_iscale, per_inst, x->sg.ctl, h_newton, 0));
  } else {
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_sg_newton_begin<<<1, 32, 0, x->stream>>>(x->st, x->sg.ctl, h_newton, 0));
  }
  HBPC_LAUNCH_CK(x, "newton graph start");
  // blocks built once per solve, at X^0 (skipped work if the loop does not run)
  if (!x->pc_every && x->sol.pc != HBPC_PC_NONE && (s = pc_build(x, x->X, c1, c2)) != HBPC_OK) return s;
  const long long r1_0 = x->stats.r1_evals, r2_0 = x->stats.r2_evals;
  B.open(h_newton, cudaGraphCondTypeWhile);
  {
    if (ni > 0) {
      if ((s = inst_scale<double>(x, x->G, nullptr, 0, nullptr)) != HBPC_OK) return s;
      if ((s = norms(x, x->G, n2)) != HBPC_OK) return s;   // of the scaled right-hand side
    }
    if (x->pc_every && x->sol.pc != HBPC_PC_NONE && (s = pc_build(x, x->X, c1, c2)) != HBPC_OK) return s;
    int kind = GM_FP64;
    if (x->sol.precision == HBPC_PREC_MIXED) {
      if ((s = to_float(x, x->X, x->Wf, n2)) != HBPC_OK) return s;
      kind = (ni > 0 && x->bk) ? GM_BATCH : GM_MIXED;
    }
    if ((s = gmres_graph(x, B, kind)) != HBPC_OK) return s;
    HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_add<<<grid_for(n2), 256, 0, x->stream>>>(x->dX, x->X, n2));
    if (ni > 0) {
      inst_sq(x->dX);
      HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_sg_save_dw_batch<<<1, 256, 0, x->stream>>>(ni, x->d_inrm, x->sg.dw));
    } else {
      if ((s = norms(x, x->dX, n2)) != HBPC_OK) return s;
      HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_sg_save_dw<<<1, 32, 0, x->stream>>>(x->st, x->sg.ctl));
    }
    if ((s = residual(x, b, c1, c2)) != HBPC_OK) return s;
    if (ni > 0) {
      inst_sq(x->G);
      HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_sg_newton_check_batch<<<1, 256, 0, x->stream>>>(ni, x->d_inrm, x->sg.dw, x->sg.g0, x->sg.active, x->d_iscale, per_inst, x->sg.ctl, h_newton, x->sol.tol_newton_rel, x->sol.tol_newton_abs, x->sol.newton_max_iter, B.own()));
    } else {
      HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_sg_newton_check<<<1, 32, 0, x->stream>>>(x->st, x->sg.ctl, h_newton, x->sol.tol_newton_rel, x->sol.tol_newton_abs, x->sol.newton_max_iter, B.own()));
    }
    HBPC_LAUNCH_CK(x, "newton graph check");
  }
  B.close();
  x->stats.r1_evals = r1_0;   // the body's evaluations are counted per iteration after the step
  x->stats.r2_evals = r2_0;
  return B.e == cudaSuccess ? HBPC_OK : cuda_fail(x, B.e, "newton graph");
}

// The configuration a step graph depends on: solver settings, operator
// parameters (passed by value into its kernels), launch shapes and buffers.
std::vector<unsigned char> step_graph_key(const hbpc_ctx* x) {
  std::vector<unsigned char> k;
  auto put = [&](const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    k.insert(k.end(), c, c + n);
  };
  put(&x->sol, sizeof(x->sol));
  put(&x->prm, sizeof(x->prm));
  put(&x->prmf, sizeof(x->prmf));
  const long long v[] = {x->nblocks, x->pc_threads, x->pc_grid, (long long)x->pc_smem, x->bk_grid, x->coop ? 1 : 0,
                         x->pc_shared ? 1 : 0, (long long)(uintptr_t)x->Jpc, (long long)(uintptr_t)x->Mpc,
                         (long long)(uintptr_t)x->Jf, (long long)(uintptr_t)x->Mf, x->s, x->pc_every};
  put(v, sizeof(v));
  return k;
}

// One step through the step graph: captured on first use and whenever the
// configuration changed, then one cudaGraphLaunch, one wait and one read of
// the control block.
hbpc_status step_graph_run(hbpc_ctx* x) {
  auto key = step_graph_key(x);
  if (!x->sg.exec || key != x->sg.key) {
    if (x->sg.exec) { cudaGraphExecDestroy(x->sg.exec); x->sg.exec = nullptr; }
    cudaGraph_t graph = nullptr;
    HBPC_CK(x, cudaGraphCreate(&graph, 0));
    const cudaStream_t real = x->stream;
    const hbpc_stats stats0 = x->stats;
    const std::string err0 = x->err;
    GBuild B{x};
    B.lv.push_back(GBuild::Level{graph, {}, x->stats.launches, 0});
    x->stream = x->sg.cap;
    x->sg.capturing = true;
    g_build = &B;
    B.begin();
    hbpc_status s = HBPC_OK;
    if (B.e == cudaSuccess) {
      HBPC_RUN(x, HBPC_PHASE_VECTOR, 1, k_sg_reset<<<1, 32, 0, x->stream>>>(x->sg.ctl));
      s = step_body(x, newton_graph, true);
    }
    B.end();
    const long long top = int(x->stats.launches - B.lv[0].l0 - B.lv[0].nested);
    x->sg.top_launches = top - 1;   // k_sg_reset counts itself on the device
    x->sg.top_r1 = x->stats.r1_evals - stats0.r1_evals;
    x->sg.top_r2 = x->stats.r2_evals - stats0.r2_evals;
    g_build = nullptr;
    x->sg.capturing = false;
    x->stream = real;
    x->stats = stats0;   // the capture ran nothing
    if (s == HBPC_OK && B.e != cudaSuccess) s = cuda_fail(x, B.e, "step graph capture");
    if (s == HBPC_OK) {
      const cudaError_t e = cudaGraphInstantiate(&x->sg.exec, graph, 0);
      if (e != cudaSuccess) { x->sg.exec = nullptr; s = cuda_fail(x, e, "step graph instantiate"); }
    }
    cudaGraphDestroy(graph);
    if (s != HBPC_OK) {
      (void)cudaGetLastError();
      return s;
    }
    x->err = err0;
    x->sg.key = key;
  }
  HBPC_CK(x, cudaGraphLaunch(x->sg.exec, x->stream));
  HBPC_CK(x, cudaMemcpyAsync(x->sg.ctl_host, x->sg.ctl, sizeof(StepCtl), cudaMemcpyDeviceToHost, x->stream));
  int sing = 0;
  if (x->singular) HBPC_CK(x, cudaMemcpyAsync(&sing, x->singular, sizeof(int), cudaMemcpyDeviceToHost, x->stream));
  hbpc_status s = sync(x, "step graph");
  if (s != HBPC_OK) return s;
  const StepCtl& c = *x->sg.ctl_host;
  const bool lin = x->ops.jv_linear != nullptr;
  const long long per = lin ? 2 : 3;
  x->stats.launches += x->sg.top_launches + c.launches;
  x->stats.newton_solves += c.newton_solves;
  x->stats.newton_its += c.newton_its;
  x->stats.gmres_its += c.gmres_its;
  x->stats.arnoldi_cols += c.arnoldi_cols;
  x->stats.r1_evals += x->sg.top_r1 + c.newton_its + c.gmres_its * (lin ? 2 : 1);
  x->stats.r2_evals += x->sg.top_r2 + c.newton_its + c.gmres_its * (per - (lin ? 2 : 1));
  if (sing) HBPC_CK(x, cudaMemsetAsync(x->singular, 0, sizeof(int), x->stream));
  // the first failure of the step (blocks built after it see its garbage)
  if (sing && !c.err) return fail(x, HBPC_ERR_NONFINITE, "BJ_ext block is singular");
  if (c.err) {
    const char* what = c.where == 1 ? "initial Newton residual is not finite"
                       : c.where == 2 ? "Newton residual is not finite"
                       : c.where == 3 ? "GMRES residual is not finite"
                                      : "Newton did not converge within newton_max_iter";
    if (c.err == HBPC_ERR_NONFINITE) return nonfinite(x, std::string("step graph: ") + what);
    return fail(x, hbpc_status(c.err), std::string("step graph: ") + what);
  }
  return HBPC_OK;
}

// Settings the step graph does not cover: the step then runs host-driven.
bool step_graph_covers(const hbpc_ctx* x) {
  return !x->schur && !x->cb && x->sol.pc != HBPC_PC_LEARNED && !x->prof.on && x->lp.per_newton == 0;
}

hbpc_status hbpc_one_step(hbpc_ctx* x) {
  if (x->sg.on && step_graph_covers(x)) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (x->stream == nullptr || (cudaStreamIsCapturing(x->stream, &cs) == cudaSuccess &&
                                 cs == cudaStreamCaptureStatusNone))
      return step_graph_run(x);
  }
  return step_body(x, newton, false);
}

template <typename Tp>
hbpc_status dmalloc(hbpc_ctx* x, Tp** p, size_t count) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(Tp));
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(x, HBPC_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  // zeroed: the padding entries between the instances of a batch are never
  // written by the operator kernels and must stay finite (they enter norms)
  e = cudaMemset(*p, 0, count * sizeof(Tp));
  if (e != cudaSuccess) return fail(x, HBPC_ERR_CUDA, std::string("cudaMemset: ") + cudaGetErrorString(e));
  return HBPC_OK;
}

void free_all(hbpc_ctx* x) {
  for (auto& g : x->arn_graph)
    if (g.exec) { cudaGraphExecDestroy(g.exec); g.exec = nullptr; }
  if (x->sg.exec) { cudaGraphExecDestroy(x->sg.exec); x->sg.exec = nullptr; }
  if (x->sg.cap) { cudaStreamDestroy(x->sg.cap); x->sg.cap = nullptr; }
  cudaFree(x->sg.ctl); cudaFree(x->sg.g0); cudaFree(x->sg.dw); cudaFree(x->sg.active);
  if (x->sg.ctl_host) cudaFreeHost(x->sg.ctl_host);
  for (auto& p : x->prof.pend) { x->prof.pool.push_back(p.a); x->prof.pool.push_back(p.b); }
  for (cudaEvent_t e : x->prof.pool) cudaEventDestroy(e);
  x->prof.pool.clear();
  x->prof.pend.clear();
  cudaFree(x->Wn); cudaFree(x->X); cudaFree(x->G); cudaFree(x->r1); cudaFree(x->r2);
  cudaFree(x->dX); cudaFree(x->bvec); cudaFree(x->stage); cudaFree(x->V); cudaFree(x->small);
  cudaFree(x->partial); cudaFree(x->ticket); cudaFree(x->st);
  cudaFree(x->kron_d); cudaFree(x->kron_f); cudaFree(x->kron_ok);
  cudaFree(x->ptc_planes); cudaFree(x->ptc_exp); cudaFree(x->ptc_err);
  cudaFree(x->sa); cudaFree(x->sb); cudaFree(x->srhs); cudaFree(x->snrm);
  cudaFree(x->Jpc); cudaFree(x->Mpc); cudaFree(x->Z); cudaFree(x->singular);
  cudaFree(x->Vf); cudaFree(x->Zf); cudaFree(x->Zf2); cudaFree(x->Wf); cudaFree(x->Mf); cudaFree(x->Jf);
  cudaFree(x->vtab_d); cudaFree(x->vtab_f); cudaFree(x->vloc_d);
  cudaFree(x->d_inst); cudaFree(x->d_instf); cudaFree(x->d_blk); cudaFree(x->d_irange);
  cudaFree(x->d_inrm); cudaFree(x->d_iscale); cudaFree(x->bk_mem);
  lp_free(x);
  if (x->st_host) cudaFreeHost(x->st_host);
}

// Launch shape of the BJ_ext apply (depends only on the block size)
void pc_launch_config(hbpc_ctx* x) {
  const int epb = std::max(1, 256 / x->nb);
  x->pc_threads = ((epb * x->nb + 31) / 32) * 32;
  x->pc_grid = int((x->nE + epb - 1) / epb);
  x->pc_smem = size_t(epb) * 4 * x->nb * sizeof(double);
}

// The tensor-core apply of the shared FP64 block: 2 n_b <= 128 (exact level
// sums) and its shared memory within the 227 KB a CTA may have.
bool ptc_fits(int nb) { return 2 * nb <= 128 && PtcDims(nb).smem() <= size_t(227 * 1024); }

// Device memory of the block preconditioners (BJ_ext and learned).
hbpc_status pc_alloc(hbpc_ctx* x) {
  if (x->Jpc) return HBPC_OK;
  const size_t blk = size_t(x->nE) * x->nb * x->nb, n2 = size_t(2 * x->ndof);
  hbpc_status e;
  if ((e = dmalloc(x, &x->Jpc, blk)) || (e = dmalloc(x, &x->Mpc, blk)) || (e = dmalloc(x, &x->Z, n2)) ||
      (e = dmalloc(x, &x->singular, 1)) || (e = dmalloc(x, &x->kron_d, 3 * kMaxP * kMaxP)) ||
      (e = dmalloc(x, &x->kron_f, 3 * kMaxP * kMaxP)) || (e = dmalloc(x, &x->kron_ok, 1)))
    return e;
  HBPC_CK(x, cudaMemsetAsync(x->singular, 0, sizeof(int), x->stream));
  if (x->phys.law == HBPC_LAW_ADVECTION && x->ptc_enable && ptc_fits(x->nb)) {
    const PtcDims D(x->nb);
    if ((e = dmalloc(x, &x->ptc_planes, D.a_bytes() / sizeof(__nv_bfloat16))) ||
        (e = dmalloc(x, &x->ptc_exp, size_t(D.R))) || (e = dmalloc(x, &x->ptc_err, 1)))
      return e;
    cudaFuncSetAttribute(k_pc_tc_planes, cudaFuncAttributeMaxDynamicSharedMemorySize, int(3 * x->nb * sizeof(double)));
    cudaFuncSetAttribute(k_pc_apply_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(D.smem()));
  }
  const size_t nbz = size_t(x->nb);
  cudaFuncSetAttribute(k_pc_form_S<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       int(nbz * nbz * sizeof(double)));
  cudaFuncSetAttribute(k_pc_invert<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       int((nbz * nbz + nbz) * sizeof(double) + nbz * sizeof(int)));
  cudaFuncSetAttribute(k_pc_form_S<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       int(nbz * nbz * sizeof(float)));
  cudaFuncSetAttribute(k_pc_invert<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       int((nbz * nbz + nbz) * sizeof(float) + nbz * sizeof(int)));
  return HBPC_OK;
}

hbpc_status pc_alloc_f(hbpc_ctx* x) {
  if (x->Mf) return HBPC_OK;
  const size_t blk = size_t(x->nE) * x->nb * x->nb;
  hbpc_status e;
  if ((e = dmalloc(x, &x->Mf, blk)) || (e = dmalloc(x, &x->Jf, blk))) return e;
  return HBPC_OK;
}

bool law_is_euler(int law) { return law == HBPC_LAW_EULER || law == HBPC_LAW_NAVIER_STOKES; }
int law_nv(int law, int dim) { return law_is_euler(law) ? dim + 2 : 1; }

hbpc_status validate(const hbpc_mesh* mesh, int N, int nodes, const hbpc_physics* ph,
                     const hbpc_solver* so) {
  auto bad = [](const std::string& m) { return fail(nullptr, HBPC_ERR_INVALID_ARG, m); };
  if (!mesh || !ph || !so) return bad("null argument");
  if (mesh->dim < 1 || mesh->dim > 3) return bad("dim must be 1, 2 or 3");
  if (mesh->periodic != 1) {
    if (mesh->periodic == 0)
      return fail(nullptr, HBPC_ERR_UNSUPPORTED, "only periodic meshes are implemented (periodic = 1)");
    return bad("periodic must be 0 or 1");
  }
  for (int m = 0; m < mesh->dim; ++m) {
    if (mesh->n[m] < 1) return bad("n[m] must be >= 1");
    if (!(mesh->hi[m] > mesh->lo[m])) return bad("hi must exceed lo");
  }
  if (N < 1 || N + 1 > kMaxP) return bad("N must satisfy 1 <= N <= 7");
  if (nodes != HBPC_NODES_LOBATTO && nodes != HBPC_NODES_GAUSS) return bad("unknown node family");
  if (ph->law < 0 || ph->law > 3) return bad("unknown law");
  if (ph->flux != HBPC_FLUX_GLOBAL_LF && ph->flux != HBPC_FLUX_RUSANOV) return bad("unknown flux");
  if (!(ph->eps > 0.0)) return bad("eps must be > 0");
  if (law_is_euler(ph->law) && !(ph->gamma > 1.0)) return bad("gamma must be > 1");
  if (std::isnan(ph->prandtl) || std::isinf(ph->prandtl)) return bad("prandtl must be finite");
  if (!(ph->nu >= 0.0) || !std::isfinite(ph->nu)) return bad("nu must be finite and >= 0");
  if (std::isnan(ph->eta_br2) || std::isinf(ph->eta_br2)) return bad("eta_br2 must be finite");
  if (ph->nu > 0.0 && ph->law == HBPC_LAW_EULER)
    return fail(nullptr, HBPC_ERR_UNSUPPORTED, "a viscous Euler flow is HBPC_LAW_NAVIER_STOKES");
  if (so->q != 4 && so->q != 6 && so->q != 8) return bad("q must be 4, 6 or 8");
  if (so->kmax < 0) return bad("kmax must be >= 0");
  if (!(so->dt > 0.0)) return bad("dt must be > 0");
  if (so->gmres_restart < 1 || so->gmres_restart > 1000) return bad("gmres_restart must be in 1..1000");
  if (so->gmres_max_iter < 1 || so->newton_max_iter < 1) return bad("iteration caps must be >= 1");
  if (!(so->tol_gmres_rel > 0.0) || !(so->tol_newton_rel >= 0.0) || !(so->tol_newton_abs >= 0.0))
    return bad("tolerances must be positive");
  if (so->pc != HBPC_PC_NONE && so->pc != HBPC_PC_BJEXT && so->pc != HBPC_PC_LEARNED && so->pc != HBPC_PC_BJEXT_H)
    return bad("unknown preconditioner");
  if (so->pc == HBPC_PC_BJEXT_H && ph->law == HBPC_LAW_NAVIER_STOKES)
    return fail(nullptr, HBPC_ERR_UNSUPPORTED, "BJ^H_ext has no Navier-Stokes Hessian blocks");
  if (so->pc != HBPC_PC_NONE) {
    int nb = law_nv(ph->law, mesh->dim);
    for (int m = 0; m < mesh->dim; ++m) nb *= (N + 1);
    if (nb > kMaxPcBlock)
      return fail(nullptr, HBPC_ERR_UNSUPPORTED, "BJ_ext block n_var (N+1)^dim exceeds the supported size");
  }
  if (so->precision != HBPC_PREC_FP64 && so->precision != HBPC_PREC_MIXED) return bad("unknown precision");
  if (!(so->t_end >= 0.0) || !std::isfinite(so->t_end)) return bad("t_end must be finite and >= 0");
  return HBPC_OK;
}

void fill_params(hbpc_ctx* x) {
  DGParams<double>& p = x->prm;
  std::memset(&p, 0, sizeof(p));
  const int P = x->P;
  for (int m = 0; m < 3; ++m) p.n[m] = m < x->dim ? x->mesh.n[m] : 1;
  p.nE = int(x->nE);
  for (int m = 0; m < x->dim; ++m) {
    // a batch keeps the matrices of h = 2 and scales by 2/h per instance
    const double h = x->ninst > 0 ? 2.0 : (x->mesh.hi[m] - x->mesh.lo[m]) / x->mesh.n[m];
    const double sc = -2.0 / h;
    // a_m folds into Dvol for inviscid advection; with a viscous term the
    // advective flux a_m w goes through the nodal-flux path instead
    const double av = (x->phys.law == HBPC_LAW_ADVECTION && !(x->phys.nu > 0.0)) ? x->phys.a[m] : 1.0;
    for (int i = 0; i < P; ++i) {
      for (int l = 0; l < P; ++l) p.Dvol[m][i][l] = sc * av * x->basis.Dhat[i * P + l];
      p.sp[m][i] = sc * x->basis.lp[i] / x->basis.w[i];
      p.sm[m][i] = sc * x->basis.lm[i] / x->basis.w[i];
    }
    for (int v = 0; v < 5; ++v) {
      double lam = 1.0;
      if (x->phys.law == HBPC_LAW_ADVECTION) lam = std::fabs(x->phys.a[m]);
      else if (law_is_euler(x->phys.law)) lam = (v == 0 || v == x->nv - 1) ? 1.0 / x->phys.eps : 1.0;
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
  // BR2 viscous term (tables on the device are attached by visc_setup)
  p.visc = x->phys.nu > 0.0 ? 1 : 0;
  p.nu = x->phys.nu;
  // Navier-Stokes (Sec. 5): mu = nu, R = 1/(gamma eps^2), c_p = R gamma/(gamma - 1),
  // lambda = c_p mu / Pr
  if (x->phys.law == HBPC_LAW_NAVIER_STOKES) {
    const double R = 1.0 / (x->phys.gamma * p.eps2);
    const double cp = R * x->phys.gamma / (x->phys.gamma - 1.0);
    const double pr = x->phys.prandtl > 0.0 ? x->phys.prandtl : 0.72;
    p.mu = x->phys.nu;
    p.kheat = cp * x->phys.nu / pr;
    p.invR = 1.0 / R;
  }
  // FP32 copy for the mixed-precision Jacobian-vector product
  DGParams<float>& f = x->prmf;
  std::memset(&f, 0, sizeof(f));
  for (int m = 0; m < 3; ++m) f.n[m] = p.n[m];
  f.nE = p.nE;
  for (int m = 0; m < 3; ++m) {
    for (int i = 0; i < kMaxP; ++i) {
      for (int l = 0; l < kMaxP; ++l) f.Dvol[m][i][l] = float(p.Dvol[m][i][l]);
      f.sp[m][i] = float(p.sp[m][i]);
      f.sm[m][i] = float(p.sm[m][i]);
    }
    for (int v = 0; v < 5; ++v) f.lam[m][v] = float(p.lam[m][v]);
    f.a[m] = float(p.a[m]);
  }
  for (int i = 0; i < kMaxP; ++i) { f.lp[i] = float(p.lp[i]); f.lm[i] = float(p.lm[i]); }
  f.gm1 = float(p.gm1); f.gamma = float(p.gamma); f.eps2 = float(p.eps2);
  f.inv_eps2 = float(p.inv_eps2); f.inv_eps = float(p.inv_eps);
  f.rusanov = p.rusanov;
  f.visc = p.visc;
  f.nu = float(p.nu);
  f.mu = float(p.mu); f.kheat = float(p.kheat); f.invR = float(p.invR);
}

// Tables of the BR2 viscous term on the device (Sec. 5.1.1): per direction the
// derivative matrix and edge derivatives scaled by 2/h (FP64 and FP32 copies)
// and the element-diagonal block used by the preconditioner assembly.
hbpc_status visc_setup(hbpc_ctx* x) {
  if (!x->prm.visc) return HBPC_OK;
  const int P = x->P, d = x->dim;
  const double eta = x->phys.eta_br2 > 0.0 ? x->phys.eta_br2 : 2.0 * d;
  const size_t ntab = size_t(d) * P * P + 2 * size_t(d) * P;
  std::vector<double> tab(ntab), vloc(size_t(d) * P * P);
  for (int m = 0; m < d; ++m) {
    const double h = x->ninst > 0 ? 2.0 : (x->mesh.hi[m] - x->mesh.lo[m]) / x->mesh.n[m];
    double bp = 0.0, bm = 0.0;
    br2_tables(x->basis, h, eta, tab.data() + size_t(m) * P * P, tab.data() + size_t(d) * P * P + m * P,
               tab.data() + size_t(d) * P * P + size_t(d) * P + m * P, &bp, &bm,
               vloc.data() + size_t(m) * P * P);
    x->prm.bp[m] = bp; x->prm.bm[m] = bm;
    x->prmf.bp[m] = float(bp); x->prmf.bm[m] = float(bm);
  }
  std::vector<float> tabf(tab.begin(), tab.end());
  hbpc_status e;
  if ((e = dmalloc(x, &x->vtab_d, ntab)) || (e = dmalloc(x, &x->vtab_f, ntab)) ||
      (e = dmalloc(x, &x->vloc_d, vloc.size())))
    return e;
  HBPC_CK(x, cudaMemcpy(x->vtab_d, tab.data(), ntab * sizeof(double), cudaMemcpyHostToDevice));
  HBPC_CK(x, cudaMemcpy(x->vtab_f, tabf.data(), ntab * sizeof(float), cudaMemcpyHostToDevice));
  HBPC_CK(x, cudaMemcpy(x->vloc_d, vloc.data(), vloc.size() * sizeof(double), cudaMemcpyHostToDevice));
  x->prm.vtab = x->vtab_d;
  x->prm.vloc = x->vloc_d;
  x->prmf.vtab = x->vtab_f;
  x->prmf.vloc = x->vloc_d;
  return HBPC_OK;
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

// Device memory and initial state of a context whose host description (sizes,
// basis, operator table, tableau, parameters) is filled in.  On failure frees
// the context and returns the error (message in g_create_error).
hbpc_status ctx_finish(hbpc_ctx* x) {
  const hbpc_solver* solver = &x->sol;
  const size_t n = size_t(x->ndof), n2 = 2 * n;
  const int m = solver->gmres_restart;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // one block per tile up to two per SM, plus one when the tiles run out first:
  // the Arnoldi column's closing block then has no rows of its own
  x->nblocks = std::max(1, std::min<int>(2 * sms, int((n2 + 1023) / 1024) + 1));
  x->nb = int(x->ndof / x->nE);
  pc_launch_config(x);
  {   // the fused CGS2 kernel needs every block resident at once
    int coop_attr = 0, per_sm_d = 0, per_sm_f = 0;
    cudaDeviceGetAttribute(&coop_attr, cudaDevAttrCooperativeLaunch, dev);
    const size_t shm_d = cgs_lowsync_smem<double>(m), shm_f = cgs_lowsync_smem<float>(m);
    if (shm_d > 48 * 1024)
      cudaFuncSetAttribute(k_cgs_lowsync<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(shm_d));
    if (shm_f > 48 * 1024)
      cudaFuncSetAttribute(k_cgs_lowsync<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(shm_f));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_d, k_cgs_lowsync<double>, kVecThreads, shm_d);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_f, k_cgs_lowsync<float>, kVecThreads, shm_f);
    cudaGetLastError();
    x->coop_max_blocks = std::min(per_sm_d, per_sm_f) * sms;
    x->coop = coop_attr && x->coop_max_blocks >= x->nblocks;
    x->sms = sms;
  }
  // partial-sum rows for every launch shape the autotuner may pick
  const int prows = std::max({x->nblocks, 4 * sms, int(x->nE)});
  // the FP64 Krylov basis only exists in the FP64 mode (the mixed mode keeps
  // two FP64 columns as scratch and its basis in FP32)
  x->vcols = solver->precision == HBPC_PREC_MIXED ? 2 : m + 1;
  hbpc_status e = HBPC_OK;
  if ((e = dmalloc(x, &x->Wn, n)) || (e = dmalloc(x, &x->X, n2)) || (e = dmalloc(x, &x->G, n2)) ||
      (e = dmalloc(x, &x->r1, n)) || (e = dmalloc(x, &x->r2, n)) || (e = dmalloc(x, &x->dX, n2)) ||
      (e = dmalloc(x, &x->bvec, n)) || (e = dmalloc(x, &x->stage, size_t(2) * x->s * 3 * n)) ||
      (e = dmalloc(x, &x->V, size_t(x->vcols) * n2))) {
    g_create_error = x->err;
    free_all(x); delete x; return e;
  }
  const size_t nsmall = size_t(m + 1) * m + 3 * m + 9 * (m + 3) + 24;
  if ((e = visc_setup(x)) != HBPC_OK) {
    g_create_error = x->err;
    free_all(x); delete x; return e;
  }
  if (solver->pc != HBPC_PC_NONE && (e = pc_alloc(x)) != HBPC_OK) {
    g_create_error = x->err;
    free_all(x); delete x; return e;
  }
  if (solver->pc == HBPC_PC_LEARNED && (e = lp_alloc(x)) != HBPC_OK) {
    g_create_error = x->err;
    free_all(x); delete x; return e;
  }
  if (solver->precision == HBPC_PREC_MIXED) {
    if ((e = dmalloc(x, &x->Vf, size_t(m + 1) * n2)) || (e = dmalloc(x, &x->Zf, n2)) ||
        (e = dmalloc(x, &x->Zf2, n2)) || (e = dmalloc(x, &x->Wf, n2))) {
      g_create_error = x->err;
      free_all(x); delete x; return e;
    }
    if (solver->pc != HBPC_PC_NONE && (e = pc_alloc_f(x)) != HBPC_OK) {
      g_create_error = x->err;
      free_all(x); delete x; return e;
    }
  }
  if ((e = dmalloc(x, &x->small, nsmall)) || (e = dmalloc(x, &x->partial, size_t(prows) * size_t(cgs_stride(m)))) ||
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
  K.hc = q; q += 2 * (m + 3);
  x->c12 = q; q += 4;
  x->dxn = q; q += 4;
  x->zn = q; q += 4;
  K.st = x->st; K.partial = x->partial; K.ticket = x->ticket; K.nblocks = x->nblocks;
  // the FP32 basis shares the small device arrays and the iteration state
  x->Kf.V = x->Vf; x->Kf.ld = K.ld; x->Kf.n2 = K.n2; x->Kf.half = K.half; x->Kf.m = K.m;
  x->Kf.H = K.H; x->Kf.cs = K.cs; x->Kf.sn = K.sn; x->Kf.g = K.g; x->Kf.vscale = K.vscale;
  x->Kf.nrmW = K.nrmW; x->Kf.nrmS = K.nrmS; x->Kf.hc = K.hc; x->Kf.y = K.y; x->Kf.st = K.st;
  x->Kf.partial = K.partial; x->Kf.ticket = K.ticket; x->Kf.nblocks = K.nblocks;
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
  return HBPC_OK;
}

// Launch-shape autotuner: times the candidates of the two runtime-shaped hot
// kernels on the context's own buffers and keeps the fastest.
//   Krylov reductions: blocks in {1, 2, 3, 4} x SMs and tiles / {1, 2, 3} (at
//     most one row tile per block, and resident all at once for the
//     cooperative CGS2 kernel); timed on CGS2 columns at j = 16 and j = m/2
//     (the state is restored afterwards).
//   Block preconditioner apply: elements per block in {1, 2, 4, 8, 16} (one
//     thread per block row, at most the 256 threads the kernel is built for).
// Every timing is the median of 7 launches after 2 warm-ups (CUDA events on
// the context's stream).  The arithmetic does not depend on the shapes except
// for the summation order of the reductions.
template <class F>
double median_us(hbpc_ctx* x, F launch) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  std::vector<float> t;
  for (int r = 0; r < 9; ++r) {
    cudaEventRecord(a, x->stream);
    launch();
    cudaEventRecord(b, x->stream);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (r >= 2) t.push_back(ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  std::sort(t.begin(), t.end());
  return 1000.0 * t[t.size() / 2];
}

hbpc_status autotune(hbpc_ctx* x, hbpc_tuning* out) {
  hbpc_status s = sync(x, "autotune");
  if (s != HBPC_OK) return s;
  const bool mixed = x->sol.precision == HBPC_PREC_MIXED;
  GmresState saved{};
  HBPC_CK(x, cudaMemcpy(&saved, x->st, sizeof(GmresState), cudaMemcpyDeviceToHost));
  // the CGS2 column is timed at two column indices, a short one (most
  // iterations of a well-preconditioned solve) and the middle of a cycle
  GmresState probe = saved;
  probe.done = 0; probe.its = 0; probe.max_its = 1 << 30; probe.m = x->sol.gmres_restart;
  probe.target = 0.0; probe.reorth = 0;
  const int jprobe[2] = {std::min(16, std::max(1, x->sol.gmres_restart - 1)),
                         std::max(1, x->sol.gmres_restart / 2)};
  GmresState* hprobe = x->st_host;           // pinned
  *hprobe = probe;
  const size_t n2 = size_t(2 * x->ndof);
  const int tiles = int((n2 + kTile - 1) / kTile);
  const int old_blocks = x->nblocks;
  double best_k = 1e300;
  int best_b = old_blocks;
  double first_k = 0.0;
  // candidates: 1..4 x SMs, and the tile count divided by 1, 2, 3 (every block
  // then gets the same number of tiles, which the grid barriers reward)
  std::vector<int> kc;
  for (int c = 1; c <= 4; ++c) kc.push_back(c * x->sms);
  for (int d = 1; d <= 3; ++d) kc.push_back((std::max(1, tiles) + d - 1) / d);
  kc.push_back(tiles + 1);   // every block one tile, plus the closing block
  for (int& v : kc) {
    v = std::min(v, std::max(1, tiles) + 1);
    if (x->coop) v = std::min(v, x->coop_max_blocks);
    v = std::max(v, 1);
  }
  std::sort(kc.begin(), kc.end());
  kc.erase(std::unique(kc.begin(), kc.end()), kc.end());
  for (int nbk : kc) {
    x->nblocks = nbk; x->K.nblocks = nbk; x->Kf.nblocks = nbk;
    double us = 0.0;
    for (int jp : jprobe) {
      hprobe->j = jp;
      us += median_us(x, [&]() {
        cudaMemcpyAsync(x->st, hprobe, sizeof(GmresState), cudaMemcpyHostToDevice, x->stream);
        if (mixed) cgs_launch<float>(x, x->Kf); else cgs_launch<double>(x, x->K);
      });
    }
    // every candidate is a launchable shape (capped by the residency check),
    // so an error here is a fault of the trial launch: stop, do not go on
    if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) {
      x->nblocks = old_blocks; x->K.nblocks = old_blocks; x->Kf.nblocks = old_blocks;
      return cuda_fail(x, e, "autotune: trial CGS2 column");
    }
    if (nbk == old_blocks) first_k = us;
    if (us < best_k) { best_k = us; best_b = nbk; }
  }
  x->nblocks = best_b; x->K.nblocks = best_b; x->Kf.nblocks = best_b;
  HBPC_LAUNCH_CK(x, "autotune krylov");
  // block preconditioner apply
  double best_p = 0.0, first_p = 0.0;
  int best_e = std::max(1, x->pc_threads / std::max(1, x->nb));
  if (x->sol.pc != HBPC_PC_NONE && (mixed ? x->Mf != nullptr : x->Mpc != nullptr)) {
    const int old_threads = x->pc_threads, old_grid = x->pc_grid;
    const size_t old_smem = x->pc_smem;
    best_p = 1e300;
    int bt = old_threads, bg = old_grid;
    size_t bs = old_smem;
    // candidates: powers of two and the creation-time shape (as many elements
    // as fit 256 threads, the kernel's launch bound)
    std::vector<int> cand = {1, 2, 4, 8, 16, std::max(1, 256 / x->nb)};
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    int last_eff = 0;
    for (int want : cand) {
      // k_pc_apply takes blockDim.x / n_b elements per block: size the grid
      // and the shared memory for that count (the thread count is rounded up
      // to whole warps)
      const int threads = ((want * x->nb + 31) / 32) * 32;
      const int epb = threads / x->nb;
      const size_t smem = size_t(epb) * 4 * x->nb * sizeof(double);
      if (threads > 256 || smem > 48 * 1024 || epb == last_eff) continue;
      last_eff = epb;
      const int grid = int((x->nE + epb - 1) / epb);
      x->pc_threads = threads; x->pc_grid = grid; x->pc_smem = smem;
      const double us = median_us(x, [&]() {
        if (mixed) pc_apply_f(x, x->Zf, nullptr, nullptr, x->Zf2, 0, nullptr);
        else pc_apply(x, x->Z, nullptr, nullptr, x->G, 0, nullptr);
      });
      if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) {
        x->pc_threads = old_threads; x->pc_grid = old_grid; x->pc_smem = old_smem;
        return cuda_fail(x, e, "autotune: trial preconditioner apply");
      }
      if (threads == old_threads) first_p = us;
      if (us < best_p) { best_p = us; bt = threads; bg = grid; bs = smem; best_e = epb; }
    }
    x->pc_threads = bt; x->pc_grid = bg; x->pc_smem = bs;
    HBPC_LAUNCH_CK(x, "autotune pc");
  }
  *hprobe = saved;
  HBPC_CK(x, cudaMemcpyAsync(x->st, hprobe, sizeof(GmresState), cudaMemcpyHostToDevice, x->stream));
  // the trial launches ran on whatever the buffers held (blocks not yet built,
  // an empty basis) and may have left non-finite values, also in the padding
  // entries of a batch that no later kernel overwrites: clear what they wrote
  const size_t n2b = size_t(2 * x->ndof);
  if (x->V) HBPC_CK(x, cudaMemsetAsync(x->V, 0, size_t(x->vcols) * n2b * sizeof(double), x->stream));
  if (x->G) HBPC_CK(x, cudaMemsetAsync(x->G, 0, n2b * sizeof(double), x->stream));
  if (x->Z) HBPC_CK(x, cudaMemsetAsync(x->Z, 0, n2b * sizeof(double), x->stream));
  if (x->Vf) HBPC_CK(x, cudaMemsetAsync(x->Vf, 0, size_t(x->sol.gmres_restart + 1) * n2b * sizeof(float), x->stream));
  if (x->Zf) HBPC_CK(x, cudaMemsetAsync(x->Zf, 0, n2b * sizeof(float), x->stream));
  if (x->Zf2) HBPC_CK(x, cudaMemsetAsync(x->Zf2, 0, n2b * sizeof(float), x->stream));
  if ((s = sync(x, "autotune")) != HBPC_OK) return s;
  if (out) {
    out->krylov_blocks = best_b;
    out->krylov_us = best_k;
    out->krylov_us_default = first_k;
    out->pc_elems_per_block = best_e;
    out->pc_us = best_p;
    out->pc_us_default = first_p;
    out->cooperative_cgs = x->coop ? 1 : 0;
  }
  return HBPC_OK;
}

// Tiles and per-instance arrays of the mixed mode's per-instance GMRES
// (batch_krylov.cuh).  Uses it when its cooperative kernel can be resident
// with a useful grid; otherwise the group keeps the shared, row-scaled GMRES.
hbpc_status bk_setup(hbpc_ctx* x) {
  const int ni = x->ninst, m = x->sol.gmres_restart;
  const long long per = x->ndof / x->nE;
  std::vector<long long> trow;
  std::vector<int> tcnt, tinst, itile;
  for (int i = 0; i < ni; ++i) {
    itile.push_back(int(tcnt.size()));
    const long long a = x->ie0[i] * per, cnt = x->inE[i] * per;
    for (int h = 0; h < 2; ++h)
      for (long long r = 0; r < cnt; r += kTile) {
        trow.push_back(h * x->ndof + a + r);
        tcnt.push_back(int(std::min<long long>(kTile, cnt - r)));
        tinst.push_back(i);
      }
  }
  itile.push_back(int(tcnt.size()));
  const int nt = int(tcnt.size());
  int per_sm = 0;
  const size_t shm = size_t(m + 1) * (kVecWarps + 1) * sizeof(double);
  if (shm > 48 * 1024)
    cudaFuncSetAttribute(k_bcgs_coop<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(shm));
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bcgs_coop<float>, kVecThreads, shm);
  int coop_attr = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&coop_attr, cudaDevAttrCooperativeLaunch, dev);
  cudaGetLastError();
  const int grid = std::min({nt, 2 * x->sms, per_sm * x->sms});
  if (!coop_attr || grid < 1) return HBPC_OK;
  // one allocation: doubles first, then the integer tables
  const size_t nd = size_t(ni) * ((m + 1) * m + 2 * m + 2 * (m + 1) + 2 * (m + 2) + 3) + size_t(nt) * (m + 3);
  const size_t bytes = nd * 8 + size_t(nt) * 8 + (size_t(nt) * 2 + (ni + 1) + 2 * ni) * 4 + 64;
  if (cudaMalloc(&x->bk_mem, bytes) != cudaSuccess) {
    x->bk_mem = nullptr;
    return fail(x, HBPC_ERR_OOM, "cudaMalloc (batched GMRES)");
  }
  char* p = static_cast<char*>(x->bk_mem);
  auto takeD = [&](size_t n) { double* r = reinterpret_cast<double*>(p); p += n * 8; return r; };
  BKrylovT<float>& K = x->BK;
  K.V = x->Vf; K.ld = size_t(2 * x->ndof); K.half = size_t(x->ndof);
  K.m = m; K.ninst = ni; K.ntiles = nt;
  K.H = takeD(size_t(ni) * (m + 1) * m);
  K.cs = takeD(size_t(ni) * m); K.sn = takeD(size_t(ni) * m);
  K.g = takeD(size_t(ni) * (m + 1)); K.y = takeD(size_t(ni) * (m + 1));
  K.hc = takeD(size_t(ni) * 2 * (m + 2));
  K.inv = takeD(ni); K.resid = takeD(ni); K.target = takeD(ni);
  K.part = takeD(size_t(nt) * (m + 3));
  long long* trow_d = reinterpret_cast<long long*>(p); p += size_t(nt) * 8;
  int* ip = reinterpret_cast<int*>(p);
  int* tcnt_d = ip; ip += nt;
  int* tinst_d = ip; ip += nt;
  int* itile_d = ip; ip += ni + 1;
  K.conv = ip; ip += ni;
  K.jn = ip; ip += ni;
  K.trow = trow_d; K.tcnt = tcnt_d; K.tinst = tinst_d; K.itile = itile_d;
  K.st = x->st;
  HBPC_CK(x, cudaMemset(x->bk_mem, 0, bytes));
  HBPC_CK(x, cudaMemcpy(trow_d, trow.data(), size_t(nt) * 8, cudaMemcpyHostToDevice));
  HBPC_CK(x, cudaMemcpy(tcnt_d, tcnt.data(), size_t(nt) * 4, cudaMemcpyHostToDevice));
  HBPC_CK(x, cudaMemcpy(tinst_d, tinst.data(), size_t(nt) * 4, cudaMemcpyHostToDevice));
  HBPC_CK(x, cudaMemcpy(itile_d, itile.data(), size_t(ni + 1) * 4, cudaMemcpyHostToDevice));
  x->bk = true;
  x->bk_grid = grid;
  return HBPC_OK;
}

// One group of a batch: the instances with the same N in one context (element
// numbering padded so that each instance starts at a multiple of the operator's
// elements per block; padding elements stay zero in every vector).
hbpc_status create_group(const std::vector<int>& ids, const hbpc_mesh* meshes, int N, int nodes,
                         const hbpc_physics* phys, const hbpc_solver* solver, hbpc_ctx** out) {
  *out = nullptr;
  hbpc_ctx* x = new (std::nothrow) hbpc_ctx();
  if (!x) return fail(nullptr, HBPC_ERR_OOM, "host allocation failed");
  const hbpc_mesh& m0 = meshes[ids[0]];
  x->mesh = m0; x->phys = phys[ids[0]]; x->sol = *solver;
  double numax = 0.0;
  for (int id : ids) numax = std::max(numax, phys[id].nu);
  x->phys.nu = numax;   // the viscous passes run if any instance is viscous
  x->N = N; x->P = N + 1; x->nodes = nodes; x->dim = m0.dim;
  x->nv = law_nv(x->phys.law, x->dim);
  long long nn = 1;
  for (int m = 0; m < x->dim; ++m) nn *= x->P;
  const int epb = nn >= 256 ? 1 : int(256 / nn);   // Geo<DIM, P>::EPB
  x->ninst = int(ids.size());
  long long e = 0;
  for (int id : ids) {
    long long ne = 1;
    for (int m = 0; m < x->dim; ++m) ne *= meshes[id].n[m];
    x->ie0.push_back(e);
    x->inE.push_back(ne);
    x->imesh.push_back(meshes[id]);
    x->inu.push_back(phys[id].nu);
    e += ((ne + epb - 1) / epb) * epb;
  }
  x->nE = e;
  x->ndof = x->nE * x->nv * nn;
  if (x->nE > (1LL << 30)) { delete x; return fail(nullptr, HBPC_ERR_INVALID_ARG, "batch too large"); }
  x->same_mesh = true;
  for (int id : ids) {
    const hbpc_mesh& mi = meshes[id];
    for (int m = 0; m < x->dim; ++m)
      if (mi.n[m] != m0.n[m] || mi.lo[m] != m0.lo[m] || mi.hi[m] != m0.hi[m]) x->same_mesh = false;
    if (phys[id].nu != phys[ids[0]].nu) x->same_mesh = false;
  }
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    delete x;
    return fail(nullptr, HBPC_ERR_CUDA, "cudaStreamCreate failed");
  }
  x->stream = st;
  if (const char* v = std::getenv("HBPC_VERBOSE")) x->verbose = std::atoi(v);
  if (const char* v = std::getenv("HBPC_GRAPH")) x->graph_mode = std::atoi(v);
  if (const char* v = std::getenv("HBPC_PC_TC")) x->ptc_enable = std::atoi(v);
  if (!basis_1d(N, nodes, x->basis) ||
      !get_ops(x->phys.law, x->dim, x->P, nodes == HBPC_NODES_LOBATTO, x->ops)) {
    cudaStreamDestroy(st);
    delete x;
    return fail(nullptr, HBPC_ERR_UNSUPPORTED, "this (law, dim, N, node family) is not compiled in");
  }
  tableau(solver->q, x);
  fill_params(x);
  hbpc_status s = ctx_finish(x);
  if (s != HBPC_OK) { cudaStreamDestroy(st); return s; }
  // instance tables
  const int ni = x->ninst;
  std::vector<InstGeo<double>> gd(ni);
  std::vector<InstGeo<float>> gf(ni);
  std::vector<long long> rng(2 * ni);
  std::vector<int> blk(size_t(x->nE / epb), 0);
  for (int i = 0; i < ni; ++i) {
    InstGeo<double>& g = gd[i];
    for (int m = 0; m < 3; ++m) g.n[m] = m < x->dim ? x->imesh[i].n[m] : 1;
    g.e0 = int(x->ie0[i]);
    g.nE = int(x->inE[i]);
    for (int m = 0; m < 3; ++m)
      g.hs[m] = m < x->dim ? 2.0 * x->imesh[i].n[m] / (x->imesh[i].hi[m] - x->imesh[i].lo[m]) : 1.0;
    g.nu = x->inu[i];
    InstGeo<float>& f = gf[i];
    for (int m = 0; m < 3; ++m) { f.n[m] = g.n[m]; f.hs[m] = float(g.hs[m]); }
    f.e0 = g.e0; f.nE = g.nE; f.nu = float(g.nu);
    rng[2 * i] = x->ie0[i] * x->nv * nn;
    rng[2 * i + 1] = x->inE[i] * x->nv * nn;
    const long long b0 = x->ie0[i] / epb, b1 = (x->ie0[i] + x->inE[i] + epb - 1) / epb;
    for (long long bb = b0; bb < b1; ++bb) blk[size_t(bb)] = i;
  }
  auto bail = [&](hbpc_status code) {
    g_create_error = x->err;
    cudaStreamDestroy(st);
    free_all(x);
    delete x;
    return code;
  };
  if ((s = dmalloc(x, &x->d_inst, ni)) || (s = dmalloc(x, &x->d_instf, ni)) || (s = dmalloc(x, &x->d_blk, blk.size())) ||
      (s = dmalloc(x, &x->d_irange, 2 * ni)) || (s = dmalloc(x, &x->d_inrm, 2 * ni)) ||
      (s = dmalloc(x, &x->d_iscale, ni)))
    return bail(s);
  cudaError_t ce = cudaMemcpy(x->d_inst, gd.data(), ni * sizeof(InstGeo<double>), cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(x->d_instf, gf.data(), ni * sizeof(InstGeo<float>), cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(x->d_blk, blk.data(), blk.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(x->d_irange, rng.data(), rng.size() * sizeof(long long), cudaMemcpyHostToDevice);
  // every vector starts at zero so that the padding elements stay zero
  const size_t n = size_t(x->ndof), n2 = 2 * n, m1 = size_t(solver->gmres_restart + 1);
  auto z = [&](void* p, size_t bytes) { if (ce == cudaSuccess && p) ce = cudaMemsetAsync(p, 0, bytes, st); };
  z(x->X, n2 * 8); z(x->G, n2 * 8); z(x->r1, n * 8); z(x->r2, n * 8); z(x->dX, n2 * 8); z(x->bvec, n * 8);
  z(x->stage, size_t(2) * x->s * 3 * n * 8); z(x->V, size_t(x->vcols) * n2 * 8); z(x->Z, n2 * 8);
  z(x->Vf, m1 * n2 * 4); z(x->Zf, n2 * 4); z(x->Zf2, n2 * 4); z(x->Wf, n2 * 4);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) { x->err = std::string("batch tables: ") + cudaGetErrorString(ce); return bail(HBPC_ERR_CUDA); }
  x->prm.inst = x->d_inst; x->prm.blk_inst = x->d_blk;
  x->prmf.inst = x->d_instf; x->prmf.blk_inst = x->d_blk;
  if (solver->precision == HBPC_PREC_MIXED && (s = bk_setup(x)) != HBPC_OK) return bail(s);
  x->h_inrm.assign(2 * ni, 0.0);
  x->h_active.assign(ni, 0);
  x->h_iscale.assign(ni, 0.0);
  *out = x;
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
  x->nv = law_nv(phys->law, mesh->dim);
  x->nE = 1;
  for (int m = 0; m < x->dim; ++m) x->nE *= mesh->n[m];
  long long nn = 1;
  for (int m = 0; m < x->dim; ++m) nn *= x->P;
  x->ndof = x->nE * x->nv * nn;
  x->stream = static_cast<cudaStream_t>(cuda_stream);
  if (const char* v = std::getenv("HBPC_VERBOSE")) x->verbose = std::atoi(v);
  if (const char* v = std::getenv("HBPC_GRAPH")) x->graph_mode = std::atoi(v);
  if (const char* v = std::getenv("HBPC_PC_TC")) x->ptc_enable = std::atoi(v);
  if (!basis_1d(N, nodes, x->basis)) { delete x; return fail(nullptr, HBPC_ERR_INVALID_ARG, "basis"); }
  if (!get_ops(phys->law, x->dim, x->P, nodes == HBPC_NODES_LOBATTO, x->ops)) {
    delete x;
    return fail(nullptr, HBPC_ERR_UNSUPPORTED, "this (law, dim, N, node family) is not compiled in");
  }
  if (x->nE > (1LL << 30)) { delete x; return fail(nullptr, HBPC_ERR_INVALID_ARG, "mesh too large"); }
  tableau(solver->q, x);
  fill_params(x);
  hbpc_status e = ctx_finish(x);
  if (e != HBPC_OK) return e;   // ctx_finish freed x
  *out = x;
  return HBPC_OK;
}

void hbpc_destroy(hbpc_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->cb) {   // runs on this context's stream, which it does not own
    free_all(ctx->cb);
    delete ctx->cb;
    ctx->cb = nullptr;
  }
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

hbpc_status hbpc_advance_to(hbpc_ctx* ctx, double t_end) {
  if (!ctx) return HBPC_ERR_INVALID_ARG;
  if (!std::isfinite(t_end)) return fail(ctx, HBPC_ERR_INVALID_ARG, "t_end must be finite");
  const double dt = ctx->sol.dt, t0 = ctx->stats.t;
  const double tol = 1e-10 * dt;
  const double span = t_end - t0;
  if (span < -tol) return fail(ctx, HBPC_ERR_INVALID_ARG, "t_end lies before the current time");
  // whole steps, then the remainder (if more than rounding of t) as one last step
  long long whole = span > 0.0 ? (long long)std::floor(span / dt) : 0;
  double rem = span - double(whole) * dt;
  if (rem > dt - tol) { whole += 1; rem = 0.0; }
  if (rem < tol) rem = 0.0;
  for (long long i = 0; i < whole; ++i) {
    hbpc_status s = hbpc_one_step(ctx);
    if (s != HBPC_OK) return s;
    ctx->stats.steps += 1;
    ctx->stats.t = t0 + double(i + 1) * dt;
  }
  if (rem > 0.0) {
    ctx->sol.dt = rem;
    hbpc_status s = hbpc_one_step(ctx);
    ctx->sol.dt = dt;
    if (s != HBPC_OK) return s;
    ctx->stats.steps += 1;
  }
  ctx->stats.t = t_end;
  return HBPC_OK;
}

hbpc_status hbpc_run(hbpc_ctx* ctx) {
  if (!ctx) return HBPC_ERR_INVALID_ARG;
  if (!(ctx->sol.t_end > 0.0)) return fail(ctx, HBPC_ERR_INVALID_ARG, "the solver has no final time t_end");
  return hbpc_advance_to(ctx, ctx->sol.t_end);
}

hbpc_status hbpc_set_wait_limit(hbpc_ctx* ctx, double seconds) {
  if (!ctx || !(seconds >= 0.0) || !std::isfinite(seconds)) return HBPC_ERR_INVALID_ARG;
  ctx->wait_limit_s = seconds;
  if (ctx->cb) ctx->cb->wait_limit_s = seconds;
  return HBPC_OK;
}

hbpc_status hbpc_set_step_graph(hbpc_ctx* ctx, int on) {
  if (!ctx || (on != 0 && on != 1)) return HBPC_ERR_INVALID_ARG;
  if (!on) {
    ctx->sg.on = false;
    return HBPC_OK;
  }
  if (ctx->schur) return fail(ctx, HBPC_ERR_UNSUPPORTED, "the step graph needs the Schur form off");
  if (ctx->cb) return fail(ctx, HBPC_ERR_UNSUPPORTED, "the step graph needs corrector batching off");
  if (ctx->sol.pc == HBPC_PC_LEARNED)
    return fail(ctx, HBPC_ERR_UNSUPPORTED, "the step graph does not cover the learned preconditioner");
  if (!ctx->sg.ctl) {
    hbpc_status s;
    if ((s = dmalloc(ctx, &ctx->sg.ctl, 1)) != HBPC_OK) return s;
    if (ctx->ninst > 0 && ((s = dmalloc(ctx, &ctx->sg.g0, ctx->ninst)) || (s = dmalloc(ctx, &ctx->sg.dw, ctx->ninst)) ||
                           (s = dmalloc(ctx, &ctx->sg.active, ctx->ninst))))
      return s;
    cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(&ctx->sg.ctl_host), sizeof(StepCtl));
    if (e != cudaSuccess) { ctx->sg.ctl_host = nullptr; return fail(ctx, HBPC_ERR_OOM, "cudaMallocHost"); }
    e = cudaStreamCreateWithFlags(&ctx->sg.cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) { ctx->sg.cap = nullptr; return cuda_fail(ctx, e, "step graph stream"); }
  }
  ctx->sg.on = true;
  return HBPC_OK;
}

hbpc_status hbpc_set_pc_rebuild(hbpc_ctx* ctx, int every_newton_iteration) {
  if (!ctx || (every_newton_iteration != 0 && every_newton_iteration != 1)) return HBPC_ERR_INVALID_ARG;
  ctx->pc_every = every_newton_iteration;
  if (ctx->cb) ctx->cb->pc_every = every_newton_iteration;
  return HBPC_OK;
}

hbpc_status hbpc_set_schur(hbpc_ctx* ctx, int on) {
  if (!ctx || (on != 0 && on != 1)) return HBPC_ERR_INVALID_ARG;
  if (!on) { ctx->schur = false; return HBPC_OK; }
  if (ctx->ninst > 0) return fail(ctx, HBPC_ERR_UNSUPPORTED, "the Schur form is for single problems");
  if (ctx->cb) return fail(ctx, HBPC_ERR_UNSUPPORTED, "the Schur form needs corrector batching off");
  if (ctx->sol.precision != HBPC_PREC_FP64)
    return fail(ctx, HBPC_ERR_UNSUPPORTED, "the Schur form is built for the FP64 mode");
  if (!ctx->sa) {
    const size_t n2 = size_t(2 * ctx->ndof);
    hbpc_status s;
    if ((s = dmalloc(ctx, &ctx->sa, n2)) || (s = dmalloc(ctx, &ctx->sb, n2)) || (s = dmalloc(ctx, &ctx->srhs, n2)) ||
        (s = dmalloc(ctx, &ctx->snrm, 4)))
      return s;
  }
  ctx->schur = true;
  return HBPC_OK;
}

// Copies the boundary description of `from` into the operator parameters of
// `to` (FP64 and FP32): the corrector-batch group of a context shares its
// boundaries.
void copy_boundaries(const hbpc_ctx* from, hbpc_ctx* to) {
  for (int m = 0; m < 3; ++m)
    for (int sd = 0; sd < 2; ++sd) {
      to->prm.bck[m][sd] = from->prm.bck[m][sd];
      to->prmf.bck[m][sd] = from->prm.bck[m][sd];
      for (int v = 0; v < 5; ++v) {
        to->prm.bcw[m][sd][v] = from->prm.bcw[m][sd][v];
        to->prmf.bcw[m][sd][v] = float(from->prm.bcw[m][sd][v]);
      }
    }
  to->bounded = from->bounded;
  to->pc_built = false;
}

hbpc_status hbpc_set_boundary(hbpc_ctx* ctx, int dir, int kind_lo, const double* state_lo, int kind_hi,
                              const double* state_hi) {
  if (!ctx) return HBPC_ERR_INVALID_ARG;
  auto bad = [&](const std::string& m) { return fail(ctx, HBPC_ERR_INVALID_ARG, m); };
  if (ctx->ninst > 0) return fail(ctx, HBPC_ERR_UNSUPPORTED, "boundaries are for single problems");
  if (dir < 0 || dir >= ctx->dim) return bad("dir must be in [0, dim)");
  const int kinds[2] = {kind_lo, kind_hi};
  const double* states[2] = {state_lo, state_hi};
  for (int sd = 0; sd < 2; ++sd)
    if (kinds[sd] != HBPC_BC_PERIODIC && kinds[sd] != HBPC_BC_DIRICHLET && kinds[sd] != HBPC_BC_WALL &&
        kinds[sd] != HBPC_BC_NOSLIP)
      return bad("unknown boundary kind");
  if ((kind_lo == HBPC_BC_PERIODIC) != (kind_hi == HBPC_BC_PERIODIC))
    return bad("a direction is periodic at both ends or at neither");
  const bool bounded = kind_lo != HBPC_BC_PERIODIC;
  if (bounded && ctx->phys.nu > 0.0 && ctx->phys.law != HBPC_LAW_NAVIER_STOKES)
    return fail(ctx, HBPC_ERR_UNSUPPORTED, "boundaries are not built for the scalar viscous term");
  double val[2][5] = {};
  for (int sd = 0; sd < 2; ++sd) {
    if (kinds[sd] == HBPC_BC_WALL && ctx->phys.law != HBPC_LAW_EULER)
      return bad("a slip wall needs the Euler equations");
    if (kinds[sd] == HBPC_BC_NOSLIP && ctx->phys.law != HBPC_LAW_NAVIER_STOKES)
      return bad("a no-slip wall needs the Navier-Stokes equations");
    if (kinds[sd] != HBPC_BC_DIRICHLET) continue;
    if (!states[sd]) return bad("a Dirichlet boundary needs its state");
    for (int v = 0; v < ctx->nv; ++v) {
      if (!std::isfinite(states[sd][v])) return bad("the Dirichlet state must be finite");
      val[sd][v] = states[sd][v];
    }
    if (law_is_euler(ctx->phys.law)) {
      const double rho = val[sd][0];
      double m2 = 0.0;
      for (int k = 0; k < ctx->dim; ++k) m2 += val[sd][1 + k] * val[sd][1 + k];
      const double eps2 = ctx->phys.eps * ctx->phys.eps;
      const double p = rho > 0.0 ? (ctx->phys.gamma - 1.0) * (val[sd][ctx->dim + 1] - 0.5 * eps2 * m2 / rho) : -1.0;
      if (!(rho > 0.0) || !(p > 0.0)) return bad("the Dirichlet state needs density and pressure > 0");
    }
  }
  hbpc_status s = sync(ctx, "set_boundary");   // no kernel of the context reads the parameters meanwhile
  if (s != HBPC_OK) return s;
  for (int sd = 0; sd < 2; ++sd) {
    ctx->prm.bck[dir][sd] = kinds[sd];
    ctx->prmf.bck[dir][sd] = kinds[sd];
    for (int v = 0; v < 5; ++v) {
      ctx->prm.bcw[dir][sd][v] = val[sd][v];
      ctx->prmf.bcw[dir][sd][v] = float(val[sd][v]);
    }
  }
  ctx->bounded = false;
  for (int m = 0; m < ctx->dim; ++m) ctx->bounded = ctx->bounded || ctx->prm.bck[m][0] != HBPC_BC_PERIODIC;
  ctx->pc_built = false;
  if (ctx->cb) copy_boundaries(ctx, ctx->cb);
  return HBPC_OK;
}

hbpc_status hbpc_set_corrector_batch(hbpc_ctx* ctx, int on) {
  if (!ctx || (on != 0 && on != 1)) return HBPC_ERR_INVALID_ARG;
  if (ctx->ninst > 0) return fail(ctx, HBPC_ERR_UNSUPPORTED, "corrector batching is for single problems");
  if (on && ctx->schur) return fail(ctx, HBPC_ERR_UNSUPPORTED, "corrector batching needs the Schur form off");
  hbpc_status s = sync(ctx, "set_corrector_batch");
  if (s != HBPC_OK) return s;
  if (!on) {
    if (ctx->cb) { free_all(ctx->cb); delete ctx->cb; ctx->cb = nullptr; }
    return HBPC_OK;
  }
  if (ctx->cb) return HBPC_OK;
  if (ctx->phys.law == HBPC_LAW_NAVIER_STOKES)
    return fail(ctx, HBPC_ERR_UNSUPPORTED, "corrector batching of the Navier-Stokes law is not built");
  if (ctx->sol.pc == HBPC_PC_LEARNED)
    return fail(ctx, HBPC_ERR_UNSUPPORTED, "corrector batching with the learned preconditioner is not built");
  const int ns = std::max(1, ctx->s - 1);
  std::vector<int> ids(ns);
  std::vector<hbpc_mesh> meshes(ns, ctx->mesh);
  std::vector<hbpc_physics> phys(ns, ctx->phys);
  for (int i = 0; i < ns; ++i) ids[i] = i;
  hbpc_ctx* g = nullptr;
  s = create_group(ids, meshes.data(), ctx->N, ctx->nodes, phys.data(), &ctx->sol, &g);
  if (s != HBPC_OK) return fail(ctx, s, std::string("corrector batch: ") + g_create_error);
  // the group works on this context's stream (its own one is released)
  cudaStreamSynchronize(g->stream);
  cudaStreamDestroy(g->stream);
  g->stream = ctx->stream;
  g->wait_limit_s = ctx->wait_limit_s;
  copy_boundaries(ctx, g);
  g->pc_every = ctx->pc_every;
  ctx->cb = g;
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
  hbpc_status s;
  if (ctx->sol.precision == HBPC_PREC_MIXED) {
    // the product the FP32 Krylov loop uses: the analytic linearisation at the
    // FP32 copy of X (dual numbers), on the FP32 direction
    if ((s = to_float(ctx, ctx->X, ctx->Wf, n2)) != HBPC_OK) return s;
    if ((s = to_float(ctx, dX, ctx->Zf, n2)) != HBPC_OK) return s;
    JvInputT<float> zf{};
    zf.V = ctx->Zf; zf.ld = n2; zf.half = size_t(n);
    zf.out = ctx->Zf2; zf.out_ld = n2; zf.out_offset = 0;
    if ((s = apply_jv_f(ctx, zf)) != HBPC_OK) return s;
    HBPC_CK(ctx, cudaMemsetAsync(out, 0, n2 * sizeof(double), ctx->stream));
    HBPC_RUN(ctx, HBPC_PHASE_VECTOR, 1, k_add_float<<<grid_for(n2), 256, 0, ctx->stream>>>(ctx->Zf2, out, n2));
    HBPC_LAUNCH_CK(ctx, "eval_Jv (mixed)");
    return sync(ctx, "eval_Jv");
  }
  HBPC_CK(ctx, cudaMemcpyAsync(ctx->dX, dX, n2 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  s = norms(ctx, ctx->dX, n2, ctx->dxn);
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
  if (ctx->sol.pc == HBPC_PC_NONE) return fail(ctx, HBPC_ERR_INVALID_ARG, "context has no preconditioner");
  const long long n = ctx->ndof;
  const size_t n2 = size_t(2 * n);
  const double dt = ctx->sol.dt;
  const double c1 = alpha1 * dt, c2 = alpha2 * dt * dt / 2.0;
  HBPC_RUN(ctx, HBPC_PHASE_VECTOR, 1, k_set2<<<1, 32, 0, ctx->stream>>>(ctx->c12, c1, c2));
  HBPC_CK(ctx, cudaMemcpyAsync(ctx->X, X, n2 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  ctx->pc_built = false;
  hbpc_status s = pc_build(ctx, ctx->X, c1, c2);
  if (s != HBPC_OK) return s;
  if (ctx->sol.precision == HBPC_PREC_MIXED) {   // the FP32 blocks and apply of the Krylov loop
    if ((s = to_float(ctx, in, ctx->Zf, n2)) != HBPC_OK) return s;
    if ((s = pc_apply_f(ctx, ctx->Zf, nullptr, nullptr, ctx->Zf2, 0, nullptr)) != HBPC_OK) return s;
    HBPC_CK(ctx, cudaMemsetAsync(out, 0, n2 * sizeof(double), ctx->stream));
    HBPC_RUN(ctx, HBPC_PHASE_VECTOR, 1, k_add_float<<<grid_for(n2), 256, 0, ctx->stream>>>(ctx->Zf2, out, n2));
    HBPC_LAUNCH_CK(ctx, "eval_pc (mixed)");
    return sync(ctx, "eval_pc");
  }
  HBPC_CK(ctx, cudaMemcpyAsync(ctx->Z, in, n2 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  if ((s = pc_apply(ctx, ctx->Z, nullptr, nullptr, out, 0, nullptr)) != HBPC_OK) return s;
  if ((s = sync(ctx, "eval_pc")) != HBPC_OK) return s;
  return ptc_check(ctx, "eval_pc");
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

hbpc_status hbpc_get_stats(const hbpc_ctx* cctx, hbpc_stats* out) {
  if (!cctx || !out) return HBPC_ERR_INVALID_ARG;
  hbpc_ctx* ctx = const_cast<hbpc_ctx*>(cctx);
  *out = ctx->stats;
  out->pc_apply_tc = ctx->ptc_ready ? 1 : 0;
  if (ctx->lp.vcount) {   // learned blocks replaced by exact inverses so far
    int v = 0;
    HBPC_CK(ctx, cudaMemcpyAsync(&v, ctx->lp.vcount, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    hbpc_status s = sync(ctx, "get_stats");
    if (s != HBPC_OK) return s;
    out->pc_exact_blocks = v - ctx->vcount_base;
  }
  return HBPC_OK;
}

hbpc_status hbpc_reset_stats(hbpc_ctx* ctx) {
  if (!ctx) return HBPC_ERR_INVALID_ARG;
  const double t = ctx->stats.t;
  ctx->stats = hbpc_stats{};
  ctx->stats.t = t;
  if (ctx->lp.vcount) {
    int v = 0;
    HBPC_CK(ctx, cudaMemcpyAsync(&v, ctx->lp.vcount, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    hbpc_status s = sync(ctx, "reset_stats");
    if (s != HBPC_OK) return s;
    ctx->vcount_base = v;
  }
  return HBPC_OK;
}

hbpc_status hbpc_set_pc(hbpc_ctx* ctx, int pc) {
  if (!ctx) return HBPC_ERR_INVALID_ARG;
  if (pc != HBPC_PC_NONE && pc != HBPC_PC_BJEXT && pc != HBPC_PC_LEARNED && pc != HBPC_PC_BJEXT_H)
    return fail(ctx, HBPC_ERR_INVALID_ARG, "unknown preconditioner");
  if (pc == HBPC_PC_BJEXT_H && ctx->phys.law == HBPC_LAW_NAVIER_STOKES)
    return fail(ctx, HBPC_ERR_UNSUPPORTED, "BJ^H_ext has no Navier-Stokes Hessian blocks");
  if (pc != HBPC_PC_NONE) {
    if (ctx->nb > kMaxPcBlock)
      return fail(ctx, HBPC_ERR_UNSUPPORTED, "block n_var (N+1)^dim exceeds the supported size");
    hbpc_status s;
    if ((s = pc_alloc(ctx)) != HBPC_OK) return s;
    if (ctx->sol.precision == HBPC_PREC_MIXED && (s = pc_alloc_f(ctx)) != HBPC_OK) return s;
    if (pc == HBPC_PC_LEARNED && (s = lp_alloc(ctx)) != HBPC_OK) return s;
  }
  if (ctx->cb) {
    if (pc == HBPC_PC_LEARNED)
      return fail(ctx, HBPC_ERR_UNSUPPORTED, "the learned preconditioner needs corrector batching off");
    hbpc_status s = hbpc_set_pc(ctx->cb, pc);
    if (s != HBPC_OK) return fail(ctx, s, "corrector batch: " + ctx->cb->err);
  }
  ctx->sol.pc = pc;
  ctx->pc_built = false;
  return HBPC_OK;
}

hbpc_status hbpc_pc_model_info(hbpc_ctx* ctx, int* d_in_padded, int* hidden, int* d_out_padded,
                               long long* n_params) {
  if (!ctx) return HBPC_ERR_INVALID_ARG;
  if (ctx->nb > kMaxPcBlock) return fail(ctx, HBPC_ERR_UNSUPPORTED, "block too large for the learned preconditioner");
  const int din = ctx->nb + 2, dinp = ((din + 15) / 16) * 16;
  const int doutp = ((ctx->nb * ctx->nb + 7) / 8) * 8, H = kMlpHidden;
  if (d_in_padded) *d_in_padded = dinp;
  if (hidden) *hidden = H;
  if (d_out_padded) *d_out_padded = doutp;
  // the layout of lp_alloc: weights and biases, standardisation, class keys and means
  if (n_params)
    *n_params = (long long)H * dinp + H + (long long)H * H + H + (long long)doutp * H + doutp + 2LL * dinp +
                2LL * kMlpClasses + (long long)kMlpClasses * doutp;
  return HBPC_OK;
}

hbpc_status hbpc_pc_model_init(hbpc_ctx* ctx, unsigned long long seed, double out_scale) {
  if (!ctx) return HBPC_ERR_INVALID_ARG;
  hbpc_status s;
  if ((s = pc_alloc(ctx)) != HBPC_OK || (s = lp_alloc(ctx)) != HBPC_OK) return s;
  auto& L = ctx->lp;
  std::vector<float> h(L.np, 0.0f);
  std::mt19937_64 rng(seed);
  std::normal_distribution<float> nd(0.0f, 1.0f);
  const size_t H = size_t(L.H);
  const float s1 = 1.0f / std::sqrt(float(L.din)), s2 = 1.0f / std::sqrt(float(H));
  for (size_t r = 0; r < H; ++r)
    for (int c = 0; c < L.din; ++c) h[L.oW1 + r * L.dinp + c] = s1 * nd(rng);
  for (size_t i = 0; i < H * H; ++i) h[L.oW2 + i] = s2 * nd(rng);
  for (int r = 0; r < L.dout; ++r)
    for (size_t c = 0; c < H; ++c) h[L.oW3 + size_t(r) * H + c] = float(out_scale) * s2 * nd(rng);
  for (int k = 0; k < L.dinp; ++k) h[L.np_train + L.dinp + k] = 1.0f;   // sd = 1, mu = 0
  HBPC_CK(ctx, cudaMemcpy(L.P, h.data(), L.np * sizeof(float), cudaMemcpyHostToDevice));
  HBPC_CK(ctx, cudaMemset(L.Mo, 0, L.np * sizeof(float)));
  HBPC_CK(ctx, cudaMemset(L.Ve, 0, L.np * sizeof(float)));
  L.adam_t = 0;
  L.stats = false;
  if ((s = lp_refresh(ctx)) != HBPC_OK) return s;
  return sync(ctx, "pc_model_init");
}

hbpc_status hbpc_pc_model_get(hbpc_ctx* ctx, float* params) {
  if (!ctx || !params || !ctx->lp.alloc) return HBPC_ERR_INVALID_ARG;
  HBPC_CK(ctx, cudaMemcpyAsync(params, ctx->lp.P, ctx->lp.np * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  return sync(ctx, "pc_model_get");
}

hbpc_status hbpc_pc_model_set(hbpc_ctx* ctx, const float* params) {
  if (!ctx || !params) return HBPC_ERR_INVALID_ARG;
  hbpc_status s;
  if ((s = pc_alloc(ctx)) != HBPC_OK || (s = lp_alloc(ctx)) != HBPC_OK) return s;
  HBPC_CK(ctx, cudaMemcpyAsync(ctx->lp.P, params, ctx->lp.np * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  ctx->lp.stats = true;   // the standardisation comes with the parameters
  if ((s = lp_refresh(ctx)) != HBPC_OK) return s;
  return sync(ctx, "pc_model_set");
}

hbpc_status hbpc_pc_loss_grad(hbpc_ctx* ctx, int loss_kind, int B, int P, const float* F, const float* J,
                              const float* c12, const float* X, double* loss, float* grads) {
  if (loss_kind != HBPC_PC_LOSS_PROBE && loss_kind != HBPC_PC_LOSS_INVERSE) return HBPC_ERR_INVALID_ARG;
  if (!ctx || !F || !J || !c12 || B < 8 || B % 8 || P < 1 || P > 16) return HBPC_ERR_INVALID_ARG;
  if (loss_kind == HBPC_PC_LOSS_PROBE && !X) return HBPC_ERR_INVALID_ARG;
  if (!ctx->lp.alloc) return fail(ctx, HBPC_ERR_INVALID_ARG, "model not initialised");
  hbpc_status s;
  if ((s = lp_alloc_train(ctx, B, P)) != HBPC_OK) return s;
  auto& L = ctx->lp;
  const size_t nf = size_t(B) * L.dinp;
  std::vector<float> ftmp(F, F + nf);
  float* dF = nullptr;
  HBPC_CK(ctx, cudaMalloc(&dF, nf * sizeof(float)));
  cudaMemcpy(dF, ftmp.data(), nf * sizeof(float), cudaMemcpyHostToDevice);
  k_f32_to_bf16<<<grid_for(nf), 256, 0, ctx->stream>>>(dF, L.Fb, nf);
  HBPC_CK(ctx, cudaMemcpyAsync(L.Jb, J, size_t(B) * L.dout * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  HBPC_CK(ctx, cudaMemcpyAsync(L.cb, c12, size_t(B) * 2 * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  if (X)
    HBPC_CK(ctx, cudaMemcpyAsync(L.Xb, X, size_t(B) * P * L.nb * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  double l = 0.0;
  s = lp_loss_grad(ctx, B, P, &l, loss_kind);
  cudaFree(dF);
  if (s != HBPC_OK) return s;
  if (loss) *loss = l;
  if (grads) {
    HBPC_CK(ctx, cudaMemcpyAsync(grads, L.G, L.np_train * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    std::fill(grads + L.np_train, grads + L.np, 0.0f);
  }
  return sync(ctx, "pc_loss_grad");
}

hbpc_status hbpc_pc_model_forward(hbpc_ctx* ctx, int B, const float* F, const float* c12, float* M) {
  if (!ctx || !F || !c12 || !M || B < 8 || B % 8) return HBPC_ERR_INVALID_ARG;
  if (!ctx->lp.alloc) return fail(ctx, HBPC_ERR_INVALID_ARG, "model not initialised");
  hbpc_status s;
  if ((s = lp_alloc_train(ctx, B, 1)) != HBPC_OK) return s;
  auto& L = ctx->lp;
  const size_t nf = size_t(B) * L.dinp;
  // the features go through the block buffer (B x n_b^2 FP32, wider than the
  // B x d_in_padded features), FP32 -> BF16 on the device
  if (nf > size_t(B) * L.dout) return fail(ctx, HBPC_ERR_UNSUPPORTED, "feature rows wider than the blocks");
  HBPC_CK(ctx, cudaMemcpyAsync(L.Jb, F, nf * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  HBPC_RUN(ctx, HBPC_PHASE_PC_BUILD, 1, k_f32_to_bf16<<<grid_for(nf), 256, 0, ctx->stream>>>(L.Jb, L.Fb, nf));
  HBPC_CK(ctx, cudaMemcpyAsync(L.cb, c12, size_t(B) * 2 * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  const int H = L.H;
  if ((s = gemm(ctx, L.Fb, L.dinp, L.W1h, L.dinp, B, H, L.dinp, EpiBiasTanh{L.P + L.ob1, L.H1b, H})) != HBPC_OK) return s;
  if ((s = gemm(ctx, L.H1b, H, L.W2h, H, B, H, H, EpiBiasTanh{L.P + L.ob2, L.H2b, H})) != HBPC_OK) return s;
  // the inference path of the preconditioner build: blocks in storage
  // (column-major) order with every row's class, then row-major for the caller
  HBPC_RUN(ctx, HBPC_PHASE_PC_BUILD, 1, k_mlp_classify<<<(B + 255) / 256, 256, 0, ctx->stream>>>(L.cb, B, L.ckey, L.cls));
  HBPC_RUN(ctx, HBPC_PHASE_PC_BUILD, 1, k_pc_bias_storage<<<grid_for(size_t(kMlpClasses) * L.doutp), 256, 0, ctx->stream>>>(L.P + L.ob3, L.cmean, kMlpClasses, L.nb, L.doutp, L.bp));
  if ((s = gemm(ctx, L.H2b, H, L.W3p, H, B, L.dout, H, EpiPcBlock<float>{L.bp, L.cls, L.doutp, L.Ob, L.nb})) != HBPC_OK)
    return s;
  HBPC_RUN(ctx, HBPC_PHASE_PC_BUILD, 1, k_blocks_to_rowmajor<<<B, 256, 0, ctx->stream>>>(L.Ob, B, L.nb, L.Jb));
  HBPC_LAUNCH_CK(ctx, "pc_model_forward");
  HBPC_CK(ctx, cudaMemcpyAsync(M, L.Jb, size_t(B) * L.dout * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  return lp_gemm_check(ctx);   // waits for the stream
}

hbpc_status hbpc_pc_adam_step(hbpc_ctx* ctx, const float* grads, double lr) {
  if (!ctx || !grads || !(lr > 0.0)) return HBPC_ERR_INVALID_ARG;
  if (!ctx->lp.alloc) return fail(ctx, HBPC_ERR_INVALID_ARG, "model not initialised");
  auto& L = ctx->lp;
  HBPC_CK(ctx, cudaMemcpyAsync(L.G, grads, L.np_train * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  L.adam_t += 1;
  const float bc1 = 1.0f - std::pow(b1, float(L.adam_t)), bc2 = 1.0f - std::pow(b2, float(L.adam_t));
  HBPC_RUN(ctx, HBPC_PHASE_PC_BUILD, 1,
           k_adam<<<grid_for(L.np_train), 256, 0, ctx->stream>>>(L.P, L.G, L.Mo, L.Ve, L.np_train, float(lr), b1, b2, eps,
                                                               bc1, bc2));
  HBPC_LAUNCH_CK(ctx, "k_adam");
  hbpc_status s = lp_refresh(ctx);
  if (s != HBPC_OK) return s;
  ctx->pc_built = false;
  return sync(ctx, "pc_adam_step");
}

hbpc_status hbpc_pc_collect(hbpc_ctx* ctx, int samples_per_newton, int capacity) {
  if (!ctx || samples_per_newton < 0 || capacity < 0) return HBPC_ERR_INVALID_ARG;
  hbpc_status s;
  if ((s = pc_alloc(ctx)) != HBPC_OK || (s = lp_alloc(ctx)) != HBPC_OK) return s;
  auto& L = ctx->lp;
  if (samples_per_newton > 0 && capacity > 0 && capacity != L.cap) {
    cudaFree(L.featbuf); cudaFree(L.Jbuf); cudaFree(L.cbuf); cudaFree(L.Tbuf);
    L.featbuf = L.Jbuf = L.cbuf = L.Tbuf = nullptr;
    if ((s = dalloc_any(ctx, &L.featbuf, size_t(capacity) * L.din)) ||
        (s = dalloc_any(ctx, &L.Jbuf, size_t(capacity) * L.dout)) ||
        (s = dalloc_any(ctx, &L.Tbuf, size_t(capacity) * L.dout)) ||
        (s = dalloc_any(ctx, &L.cbuf, size_t(capacity) * 2)))
      return s;
    L.cap = capacity; L.count = 0; L.next = 0; L.targets = true;
  }
  if (samples_per_newton > 0 && L.cap == 0) return fail(ctx, HBPC_ERR_INVALID_ARG, "capacity must be > 0");
  L.per_newton = samples_per_newton;
  return HBPC_OK;
}

hbpc_status hbpc_pc_train(hbpc_ctx* ctx, int loss_kind, int iters, int batch, int probes, double lr,
                          unsigned long long seed, double* loss_first, double* loss_last) {
  if (!ctx || iters < 1 || batch < 8 || batch % 8 || probes < 1 || probes > 16 || !(lr > 0.0))
    return HBPC_ERR_INVALID_ARG;
  if (loss_kind != HBPC_PC_LOSS_PROBE && loss_kind != HBPC_PC_LOSS_INVERSE) return HBPC_ERR_INVALID_ARG;
  auto& L = ctx->lp;
  if (!L.alloc) return fail(ctx, HBPC_ERR_INVALID_ARG, "model not initialised");
  if (L.count < batch) return fail(ctx, HBPC_ERR_INVALID_ARG, "replay buffer holds fewer samples than a batch");
  if (loss_kind == HBPC_PC_LOSS_INVERSE && !(L.Tbuf && L.targets))
    return fail(ctx, HBPC_ERR_INVALID_ARG, "inverse regression needs data collected with the BJ_ext preconditioner");
  hbpc_status s;
  if ((s = lp_alloc_train(ctx, batch, probes)) != HBPC_OK) return s;
  if (!L.stats) {   // feature standardisation from the replay buffer
    std::vector<float> f(size_t(L.count) * L.din);
    HBPC_CK(ctx, cudaMemcpy(f.data(), L.featbuf, f.size() * sizeof(float), cudaMemcpyDeviceToHost));
    std::vector<float> mu(L.dinp, 0.0f), sd(L.dinp, 1.0f);
    for (int k = 0; k < L.din; ++k) {
      double m = 0.0, q = 0.0;
      for (int i = 0; i < L.count; ++i) m += f[size_t(i) * L.din + k];
      m /= L.count;
      for (int i = 0; i < L.count; ++i) { const double d = f[size_t(i) * L.din + k] - m; q += d * d; }
      const double sdv = std::sqrt(q / L.count);
      mu[k] = float(m);
      sd[k] = sdv > 1e-6 * (std::fabs(m) + 1e-30) && sdv > 0.0 ? float(sdv) : 1.0f;
    }
    HBPC_CK(ctx, cudaMemcpy(L.mu, mu.data(), L.dinp * sizeof(float), cudaMemcpyHostToDevice));
    HBPC_CK(ctx, cudaMemcpy(L.sd, sd.data(), L.dinp * sizeof(float), cudaMemcpyHostToDevice));
    // stage classes: the first kMlpClasses distinct (c1, c2) pairs of the buffer
    std::vector<float> cb(size_t(L.count) * 2);
    HBPC_CK(ctx, cudaMemcpy(cb.data(), L.cbuf, cb.size() * sizeof(float), cudaMemcpyDeviceToHost));
    std::vector<float> keys(2 * kMlpClasses, -1.0f);
    int nk = 0;
    for (int i = 0; i < L.count && nk < kMlpClasses; ++i) {
      bool seen = false;
      for (int k = 0; k < nk; ++k) seen = seen || (keys[2 * k] == cb[2 * i] && keys[2 * k + 1] == cb[2 * i + 1]);
      if (!seen) { keys[2 * nk] = cb[2 * i]; keys[2 * nk + 1] = cb[2 * i + 1]; ++nk; }
    }
    HBPC_CK(ctx, cudaMemcpy(L.ckey, keys.data(), keys.size() * sizeof(float), cudaMemcpyHostToDevice));
    HBPC_CK(ctx, cudaMemset(L.cmean, 0, size_t(kMlpClasses) * L.doutp * sizeof(float)));
    if (L.Tbuf && L.targets)   // each class starts from its mean block inverse
      for (int k = 0; k < nk; ++k)
        k_mlp_class_mean<<<(L.dout + 255) / 256, 256, 0, ctx->stream>>>(L.Tbuf, L.cbuf, L.count, L.nb, keys[2 * k],
                                                                        keys[2 * k + 1], L.cmean + size_t(k) * L.doutp);
    HBPC_LAUNCH_CK(ctx, "class means");
    L.stats = true;
  }
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int it = 0; it < iters; ++it) {
    const unsigned long long sd = seed * 1000003ull + unsigned(it);
    HBPC_RUN(ctx, HBPC_PHASE_PC_BUILD, 1, k_rand_idx<<<(batch + 255) / 256, 256, 0, ctx->stream>>>(L.idx, batch, L.count, sd));
    HBPC_RUN(ctx, HBPC_PHASE_PC_BUILD, 1,
             k_mlp_gather<<<batch, 128, 0, ctx->stream>>>(L.featbuf, loss_kind == HBPC_PC_LOSS_INVERSE ? L.Tbuf : L.Jbuf,
                                                           L.cbuf, L.idx, batch, L.din, L.dinp, L.nb,
                                                           L.mu, L.sd, L.Fb, L.Jb, L.cb));
    const size_t nx = size_t(batch) * probes * L.nb;
    HBPC_RUN(ctx, HBPC_PHASE_PC_BUILD, 1, k_rademacher<<<grid_for(nx), 256, 0, ctx->stream>>>(L.Xb, nx, sd + 17));
    HBPC_LAUNCH_CK(ctx, "pc_train sample");
    double l = 0.0;
    const bool want = (it == 0 && loss_first) || (it == iters - 1 && loss_last);
    if ((s = lp_loss_grad(ctx, batch, probes, want ? &l : nullptr, loss_kind)) != HBPC_OK) return s;
    if (it == 0 && loss_first) *loss_first = l;
    if (it == iters - 1 && loss_last) *loss_last = l;
    L.adam_t += 1;
    const float bc1 = 1.0f - std::pow(b1, float(L.adam_t)), bc2 = 1.0f - std::pow(b2, float(L.adam_t));
    HBPC_RUN(ctx, HBPC_PHASE_PC_BUILD, 1,
             k_adam<<<grid_for(L.np_train), 256, 0, ctx->stream>>>(L.P, L.G, L.Mo, L.Ve, L.np_train, float(lr), b1, b2, eps, bc1, bc2));
    HBPC_LAUNCH_CK(ctx, "k_adam");
    if ((s = lp_refresh(ctx)) != HBPC_OK) return s;
  }
  ctx->pc_built = false;
  return lp_gemm_check(ctx);   // waits for the stream
}

hbpc_status hbpc_profile_enable(hbpc_ctx* ctx, int enable) {
  if (!ctx) return HBPC_ERR_INVALID_ARG;
  hbpc_status s = sync(ctx, "profile_enable");
  if (s != HBPC_OK) return s;
  ctx->prof.on = enable != 0;
  for (int i = 0; i < HBPC_NPHASES; ++i) { ctx->prof.ms[i] = 0.0; ctx->prof.cnt[i] = 0; }
  if (ctx->cb) return hbpc_profile_enable(ctx->cb, enable);
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
  if (ctx->cb) {   // the batched correctors' launches
    if ((s = sync(ctx->cb, "profile_get")) != HBPC_OK) return s;
    for (int i = 0; i < n_phases && i < HBPC_NPHASES; ++i) {
      if (ms) ms[i] += ctx->cb->prof.ms[i];
      if (launches) launches[i] += ctx->cb->prof.cnt[i];
    }
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
  if (phys->nu != 0.0)
    return fail(nullptr, HBPC_ERR_UNSUPPORTED, "the allocation-free Jv has no viscous term; use hbpc_eval_Jv");
  // host-side description of the discretisation (no device memory)
  hbpc_ctx x;
  x.mesh = *mesh; x.phys = *phys; x.sol = so;
  x.N = N; x.P = N + 1; x.nodes = nodes; x.dim = mesh->dim;
  x.nv = law_nv(phys->law, mesh->dim);
  x.nE = 1;
  for (int m = 0; m < x.dim; ++m) x.nE *= mesh->n[m];
  long long nn = 1;
  for (int m = 0; m < x.dim; ++m) nn *= x.P;
  x.ndof = x.nE * x.nv * nn;
  if (x.ndof > kNoAllocMaxDof)
    return fail(nullptr, HBPC_ERR_INVALID_ARG,
                "n_dof exceeds the allocation-free limit of 262144 values; use hbpc_eval_Jv");
  {
    // out is written while X and dX are still being read: no overlap allowed
    const uintptr_t len = uintptr_t(2 * x.ndof) * sizeof(double);
    auto overlaps = [&](const void* a, const void* b) {
      const uintptr_t pa = reinterpret_cast<uintptr_t>(a), pb = reinterpret_cast<uintptr_t>(b);
      return pa < pb + len && pb < pa + len;
    };
    if (overlaps(out, X) || overlaps(out, dX))
      return fail(nullptr, HBPC_ERR_INVALID_ARG, "out overlaps X or dX; pass a separate output array");
  }
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
  // after the first enqueue an error still waits for the stream, so that no
  // work of a failed call is left running on the shared array
  auto ck = [&](cudaError_t e, const char* what) -> hbpc_status {
    if (e == cudaSuccess) return HBPC_OK;
    cudaStreamSynchronize(stream);
    return cuda_fail(nullptr, e, what);
  };
  // the shared array keeps the previous call's contents: the ticket must start at 0
  if ((st = ck(cudaMemsetAsync(K.ticket, 0, sizeof(unsigned), stream), "clear ticket")) != HBPC_OK) return st;
  k_set2<<<1, 32, 0, stream>>>(c12, c1, c2);
  // R1(W), R2(W, S) at X into the scratch (G goes to `out`, overwritten below)
  x.ops.residual(x.prm, X, X + n, X, c1, c2, out, out + n, scr + kNoAllocR1, scr + kNoAllocR2, stream);
  k_norms<double, double><<<K.nblocks, kVecThreads, 0, stream>>>(dX, n2, size_t(n), K, nullptr);
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

/* ---- batches of independent instances ---------------------------------- */
hbpc_status hbpc_batch_create(hbpc_batch** out, int n_inst, const hbpc_mesh* meshes, const int* N, int nodes,
                              const hbpc_physics* phys, const hbpc_solver* solver, int max_per_group) {
  if (!out || n_inst < 1 || !meshes || !N || !phys || !solver)
    return fail(nullptr, HBPC_ERR_INVALID_ARG, "invalid batch arguments");
  *out = nullptr;
  for (int i = 0; i < n_inst; ++i) {
    hbpc_status s = validate(&meshes[i], N[i], nodes, &phys[i], solver);
    if (s != HBPC_OK) return s;
    if (phys[i].law == HBPC_LAW_NAVIER_STOKES)
      return fail(nullptr, HBPC_ERR_UNSUPPORTED, "batches of the Navier-Stokes law are not supported");
    const hbpc_physics& a = phys[0];
    const hbpc_physics& b = phys[i];
    if (b.law != a.law || b.flux != a.flux || b.gamma != a.gamma || b.eps != a.eps || b.lf_scale != a.lf_scale ||
        b.a[0] != a.a[0] || b.a[1] != a.a[1] || b.a[2] != a.a[2] || b.eta_br2 != a.eta_br2 ||
        meshes[i].dim != meshes[0].dim)
      return fail(nullptr, HBPC_ERR_INVALID_ARG,
                  "batch instances must share dim, law, flux, gamma, eps, lf_scale, a and eta_br2");
  }
  if (solver->pc == HBPC_PC_LEARNED)
    return fail(nullptr, HBPC_ERR_UNSUPPORTED, "the learned preconditioner is not available for batches");
  hbpc_batch* b = new (std::nothrow) hbpc_batch();
  if (!b) return fail(nullptr, HBPC_ERR_OOM, "host allocation failed");
  b->ig.assign(n_inst, -1);
  b->il.assign(n_inst, -1);
  const int cap = max_per_group > 0 ? max_per_group : n_inst;
  for (int Nv = 1; Nv <= kMaxP - 1; ++Nv) {
    std::vector<int> all;
    for (int i = 0; i < n_inst; ++i)
      if (N[i] == Nv) all.push_back(i);
    // instances of one N in groups of at most `cap`, sizes sorted so that a
    // group holds instances of similar size
    std::stable_sort(all.begin(), all.end(), [&](int a, int c) {
      long long na = 1, nc = 1;
      for (int m = 0; m < meshes[a].dim; ++m) { na *= meshes[a].n[m]; nc *= meshes[c].n[m]; }
      return na < nc;
    });
    for (size_t g0 = 0; g0 < all.size(); g0 += size_t(cap)) {
      std::vector<int> ids(all.begin() + g0, all.begin() + std::min(all.size(), g0 + size_t(cap)));
      hbpc_ctx* x = nullptr;
      hbpc_status s = create_group(ids, meshes, Nv, nodes, phys, solver, &x);
      if (s != HBPC_OK) { hbpc_batch_destroy(b); return s; }
      for (size_t k = 0; k < ids.size(); ++k) { b->ig[ids[k]] = int(b->g.size()); b->il[ids[k]] = int(k); }
      b->g.push_back(x);
    }
  }
  *out = b;
  return HBPC_OK;
}

void hbpc_batch_destroy(hbpc_batch* b) {
  if (!b) return;
  for (hbpc_ctx* x : b->g) {
    cudaStreamSynchronize(x->stream);
    cudaStream_t st = x->stream;
    hbpc_destroy(x);
    cudaStreamDestroy(st);
  }
  delete b;
}

int hbpc_batch_groups(const hbpc_batch* b) { return b ? int(b->g.size()) : 0; }

long long hbpc_batch_ndof(const hbpc_batch* b, int inst) {
  if (!b || inst < 0 || inst >= int(b->ig.size())) return -1;
  const hbpc_ctx* x = b->g[b->ig[inst]];
  return x->inE[b->il[inst]] * (x->ndof / x->nE);
}

static hbpc_status batch_inst(hbpc_batch* b, int inst, hbpc_ctx** x, size_t* off, size_t* cnt) {
  if (!b || inst < 0 || inst >= int(b->ig.size())) return HBPC_ERR_INVALID_ARG;
  *x = b->g[b->ig[inst]];
  const int k = b->il[inst];
  const size_t per = size_t((*x)->ndof / (*x)->nE);
  *off = size_t((*x)->ie0[k]) * per;
  *cnt = size_t((*x)->inE[k]) * per;
  return HBPC_OK;
}

hbpc_status hbpc_batch_set_state(hbpc_batch* b, int inst, const double* w, int on_device) {
  hbpc_ctx* x; size_t off, cnt;
  if (!w || batch_inst(b, inst, &x, &off, &cnt) != HBPC_OK) return HBPC_ERR_INVALID_ARG;
  HBPC_CK(x, cudaMemcpyAsync(x->Wn + off, w, cnt * sizeof(double),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, x->stream));
  return sync(x, "batch set_state");
}

hbpc_status hbpc_batch_get_state(hbpc_batch* b, int inst, double* w, int on_device) {
  hbpc_ctx* x; size_t off, cnt;
  if (!w || batch_inst(b, inst, &x, &off, &cnt) != HBPC_OK) return HBPC_ERR_INVALID_ARG;
  HBPC_CK(x, cudaMemcpyAsync(w, x->Wn + off, cnt * sizeof(double),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, x->stream));
  return sync(x, "batch get_state");
}

hbpc_status hbpc_batch_node_coords(hbpc_batch* b, int inst, double* xo) {
  hbpc_ctx* x; size_t off, cnt;
  if (!xo || batch_inst(b, inst, &x, &off, &cnt) != HBPC_OK) return HBPC_ERR_INVALID_ARG;
  const int k = b->il[inst];
  const hbpc_mesh& mesh = x->imesh[k];
  const int d = x->dim, P = x->P;
  long long nn = 1;
  for (int m = 0; m < d; ++m) nn *= P;
  const long long nE = x->inE[k], per = nE * nn;
  for (long long e = 0; e < nE; ++e) {
    long long ec[3] = {0, 0, 0};
    ec[0] = e % mesh.n[0];
    if (d > 1) ec[1] = (e / mesh.n[0]) % mesh.n[1];
    if (d > 2) ec[2] = e / (mesh.n[0] * (long long)mesh.n[1]);
    for (long long node = 0; node < nn; ++node) {
      long long id[3] = {node % P, (node / P) % P, node / (P * P)};
      for (int m = 0; m < d; ++m) {
        const double h = (mesh.hi[m] - mesh.lo[m]) / mesh.n[m];
        xo[m * per + e * nn + node] = mesh.lo[m] + h * ec[m] + 0.5 * h * (x->basis.xi[id[m]] + 1.0);
      }
    }
  }
  return HBPC_OK;
}

hbpc_status hbpc_batch_eval_R1(hbpc_batch* b, int inst, double* r) {
  hbpc_ctx* x; size_t off, cnt;
  if (!r || batch_inst(b, inst, &x, &off, &cnt) != HBPC_OK) return HBPC_ERR_INVALID_ARG;
  HBPC_RUN(x, HBPC_PHASE_OPERATOR, 1, x->ops.r1(x->prm, x->Wn, x->r1, x->stream));
  HBPC_LAUNCH_CK(x, "batch eval_R1");
  HBPC_CK(x, cudaMemcpyAsync(r, x->r1 + off, cnt * sizeof(double), cudaMemcpyDeviceToHost, x->stream));
  return sync(x, "batch eval_R1");
}

hbpc_status hbpc_batch_set_pc_rebuild(hbpc_batch* b, int every_newton_iteration) {
  if (!b || (every_newton_iteration != 0 && every_newton_iteration != 1)) return HBPC_ERR_INVALID_ARG;
  for (hbpc_ctx* x : b->g) x->pc_every = every_newton_iteration;
  return HBPC_OK;
}

hbpc_status hbpc_batch_set_step_graph(hbpc_batch* b, int on) {
  if (!b || (on != 0 && on != 1)) return HBPC_ERR_INVALID_ARG;
  for (hbpc_ctx* x : b->g) {
    const hbpc_status s = hbpc_set_step_graph(x, on);
    if (s != HBPC_OK) { b->err = x->err; return s; }
  }
  return HBPC_OK;
}

hbpc_status hbpc_batch_step(hbpc_batch* b, int n_steps) {
  if (!b || n_steps < 0) return HBPC_ERR_INVALID_ARG;
  const size_t G = b->g.size();
  std::vector<hbpc_status> st(G, HBPC_OK);
  if (G == 1) {
    st[0] = hbpc_step(b->g[0], n_steps);
  } else {
    // one host thread per group, each on its group's stream
    std::vector<std::thread> th;
    th.reserve(G);
    for (size_t k = 0; k < G; ++k) th.emplace_back([&, k]() { st[k] = hbpc_step(b->g[k], n_steps); });
    for (auto& t : th) t.join();
  }
  for (size_t k = 0; k < G; ++k)
    if (st[k] != HBPC_OK) { b->err = b->g[k]->err; return st[k]; }
  return HBPC_OK;
}

hbpc_status hbpc_batch_get_stats(const hbpc_batch* b, hbpc_stats* out) {
  if (!b || !out) return HBPC_ERR_INVALID_ARG;
  hbpc_stats t{};
  for (const hbpc_ctx* x : b->g) {
    t.steps = std::max(t.steps, x->stats.steps);
    t.newton_solves += x->stats.newton_solves;
    t.newton_its += x->stats.newton_its;
    t.gmres_its += x->stats.gmres_its;
    t.r1_evals += x->stats.r1_evals;
    t.r2_evals += x->stats.r2_evals;
    t.launches += x->stats.launches;
    t.arnoldi_cols += x->stats.arnoldi_cols;
    t.t = std::max(t.t, x->stats.t);
  }
  *out = t;
  return HBPC_OK;
}

hbpc_status hbpc_autotune(hbpc_ctx* ctx, hbpc_tuning* out) {
  if (!ctx) return HBPC_ERR_INVALID_ARG;
  if (ctx->cb) {   // the corrector batch has its own vector lengths
    hbpc_status s = autotune(ctx->cb, nullptr);
    if (s != HBPC_OK) return fail(ctx, s, "corrector batch: " + ctx->cb->err);
  }
  return autotune(ctx, out);
}

hbpc_status hbpc_batch_autotune(hbpc_batch* b, hbpc_tuning* out, int n_out) {
  if (!b || (out && n_out < int(b->g.size()))) return HBPC_ERR_INVALID_ARG;
  for (size_t k = 0; k < b->g.size(); ++k) {
    hbpc_status s = autotune(b->g[k], out ? out + k : nullptr);
    if (s != HBPC_OK) { b->err = b->g[k]->err; return s; }
  }
  return HBPC_OK;
}

hbpc_status hbpc_batch_profile_enable(hbpc_batch* b, int enable) {
  if (!b) return HBPC_ERR_INVALID_ARG;
  for (hbpc_ctx* x : b->g) {
    hbpc_status s = hbpc_profile_enable(x, enable);
    if (s != HBPC_OK) return s;
  }
  return HBPC_OK;
}

const char* hbpc_batch_last_error(const hbpc_batch* b) {
  if (!b) return g_create_error.c_str();
  return b->err.c_str();
}

const char* hbpc_last_error(const hbpc_ctx* ctx) {
  if (!ctx) return g_create_error.c_str();
  return ctx->err.c_str();
}

}  // extern "C"
