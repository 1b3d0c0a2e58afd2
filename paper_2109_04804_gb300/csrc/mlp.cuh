// Learned block preconditioner: a per-element multilayer perceptron
//   f_e = standardised [W_e (n_b values), c1, c2]        (features, padded to d_inp)
//   h1 = tanh(W1 f + b1), h2 = tanh(W2 h1 + b2), O = W3 h2 + b3,  M~_e = I + reshape(O)
// that replaces the inverse M_e = S_e^-1 of the BJ_ext block S = I - c1 J + c2 J^2
// (Sec. 3.2.3) in the preconditioner apply, and its training with the probe
// loss  L = sum_{e,p} || M~_e S_e x_p - x_p ||^2 / (B P)  on (features, J_e)
// samples collected from the method's own Newton iterations.  The paper has no
// learned preconditioner; the same Newton tolerance fixes the answer whatever
// preconditioner is used.
//
// GEMMs: BF16 operands, FP32 accumulation on tcgen05 (gemm_tc.cuh); master weights,
// Adam moments and the probe arithmetic in FP32.  Included by one translation
// unit.
#pragma once
#include <cuda_bf16.h>

#include "gemm_tc.cuh"

namespace hbpc {

constexpr int kMlpHidden = 256;
constexpr int kMlpClasses = 4;   // stage classes: distinct (c1, c2) pairs with their own mean inverse

// Class of a stage coefficient pair: the key equal to (c1, c2), else the
// nearest in relative distance (keys with c1 <= 0 are unused).
__device__ __host__ inline int mlp_class(const float* keys, float c1, float c2) {
  int best = 0;
  float bd = 3.0e38f;
  for (int k = 0; k < kMlpClasses; ++k) {
    const float k1 = keys[2 * k], k2 = keys[2 * k + 1];
    if (!(k1 > 0.f)) continue;
    if (k1 == c1 && k2 == c2) return k;
    const float d = fabsf(c1 - k1) / k1 + fabsf(c2 - k2) / fmaxf(fabsf(k2), 1e-30f);
    if (d < bd) { bd = d; best = k; }
  }
  return best;
}

// ---- epilogues ---------------------------------------------------------------
struct EpiBiasTanh {            // out = bf16(tanh(acc + b[n]))
  const float* b; __nv_bfloat16* out; int ld;
  __device__ void operator()(int m, int n, float acc) const {
    out[size_t(m) * ld + n] = __float2bfloat16(tanhf(acc + b[n]));
  }
};
struct EpiBiasF32 {             // out = acc + b[n]
  const float* b; float* out; int ld;
  __device__ void operator()(int m, int n, float acc) const { out[size_t(m) * ld + n] = acc + b[n]; }
};
struct EpiStore {               // out = acc
  float* out; int ld;
  __device__ void operator()(int m, int n, float acc) const { out[size_t(m) * ld + n] = acc; }
};
struct EpiDtanh {               // out = bf16(acc * (1 - h^2)), h the layer's activation
  const __nv_bfloat16* H; __nv_bfloat16* out; int ld;
  __device__ void operator()(int m, int n, float acc) const {
    const float h = __bfloat162float(H[size_t(m) * ld + n]);
    out[size_t(m) * ld + n] = __float2bfloat16(acc * (1.f - h * h));
  }
};
// M~ of element m = I + C_k + reshape(acc + b), C_k the mean block inverse
// (minus I) of the element's stage class k: network output n = r nb + c is
// entry (r, c).  The GEMM runs with the rows of W3 permuted (W3p, from
// k_w3_permute) so that its output column p = c nb + r is already the
// column-major storage position of entry (r, c) in the element's block, and
// bias, class mean and identity come pre-permuted (k_pc_bias_storage): the 16
// accumulator values a thread holds become 16 consecutive floats (doubles) of
// one block, read and written with 16-byte accesses.
template <typename S>
struct EpiPcBlock {
  static constexpr bool kStore16 = true;
  const float* bp;   // per class: bias + class mean + identity in storage order (k_pc_bias_storage)
  const int* cls;    // class of every row, or null: one class (bp is its row)
  int doutp; S* M; int nb;
  __device__ __forceinline__ const float* row_bias(int m) const { return cls ? bp + size_t(cls[m]) * doutp : bp; }
  __device__ void operator()(int m, int p, float acc) const {
    M[size_t(m) * nb * nb + p] = S(acc + row_bias(m)[p]);
  }
  // columns p0 .. p0 + 15 of row m (those < N), accumulators as raw FP32 bits
  __device__ void store16(int m, int p0, const uint32_t* acc, int N) const {
    const float* bb = row_bias(m) + p0;
    S* dst = M + size_t(m) * nb * nb + p0;
    if (p0 + 16 <= N && (reinterpret_cast<uintptr_t>(dst) & 15) == 0 && (reinterpret_cast<uintptr_t>(bb) & 15) == 0) {
      S v[16];
#pragma unroll
      for (int q = 0; q < 16; q += 4) {
        const float4 b4 = *reinterpret_cast<const float4*>(bb + q);
        v[q] = S(__uint_as_float(acc[q]) + b4.x);
        v[q + 1] = S(__uint_as_float(acc[q + 1]) + b4.y);
        v[q + 2] = S(__uint_as_float(acc[q + 2]) + b4.z);
        v[q + 3] = S(__uint_as_float(acc[q + 3]) + b4.w);
      }
      constexpr int per = 16 / sizeof(S);
#pragma unroll
      for (int q = 0; q < 16; q += per) *reinterpret_cast<uint4*>(dst + q) = *reinterpret_cast<const uint4*>(v + q);
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (p0 + j < N) dst[j] = S(__uint_as_float(acc[j]) + bb[j]);
    }
  }
};

// out[k][p] = b[n] + cm[k][n] + (r == c) for the classes k < ncls, p = c nb + r
// the storage position of entry (r, c), n = r nb + c its network output
// (rows of doutp floats; padding zero).
__global__ void k_pc_bias_storage(const float* __restrict__ b, const float* __restrict__ cm, int ncls, int nb,
                                  int doutp, float* __restrict__ out) {
  const size_t total = size_t(ncls) * doutp;
  for (size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += size_t(gridDim.x) * blockDim.x) {
    const int k = int(t / doutp), p = int(t - size_t(k) * doutp);
    if (p >= nb * nb) { out[t] = 0.f; continue; }
    const int c = p / nb, r = p - c * nb, n = r * nb + c;
    out[t] = b[n] + cm[size_t(k) * doutp + n] + (r == c ? 1.f : 0.f);
  }
}

// W3p row p = W3 row n(p), n(p) = (p mod nb) nb + p div nb for p < nb^2 (the
// storage order of the blocks, see EpiPcBlock); padding rows zero.
__global__ void k_w3_permute(const __nv_bfloat16* __restrict__ W3, __nv_bfloat16* __restrict__ W3p, int nb,
                             int doutp, int H) {
  const size_t total = size_t(doutp) * H;
  for (size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += size_t(gridDim.x) * blockDim.x) {
    const int p = int(t / H), k = int(t - size_t(p) * H);
    if (p >= nb * nb) { W3p[t] = __float2bfloat16(0.f); continue; }
    const int n = (p % nb) * nb + p / nb;
    W3p[t] = W3[size_t(n) * H + k];
  }
}

// Column-major blocks (the storage order) to row-major ones, B blocks of nb^2.
__global__ void k_blocks_to_rowmajor(const float* __restrict__ in, int B, int nb, float* __restrict__ out) {
  const int e = blockIdx.x;
  if (e >= B) return;
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int i = t / nb, j = t - i * nb;
    out[size_t(e) * nb * nb + t] = in[size_t(e) * nb * nb + size_t(j) * nb + i];
  }
}

// ---- small kernels ----------------------------------------------------------
// Features of every element: standardised state and stage coefficients.
__global__ void k_mlp_features(const double* __restrict__ W, int nE, int nb, double c1, double c2,
                               const float* __restrict__ mu, const float* __restrict__ sd, int dinp,
                               __nv_bfloat16* __restrict__ F) {
  const size_t total = size_t(nE) * dinp;
  for (size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += size_t(gridDim.x) * blockDim.x) {
    const int e = int(t / dinp), k = int(t - size_t(e) * dinp);
    float v = 0.f;
    if (k < nb) v = float(W[size_t(e) * nb + k]);
    else if (k == nb) v = float(c1);
    else if (k == nb + 1) v = float(c2);
    v = (k < nb + 2) ? (v - mu[k]) / sd[k] : 0.f;
    F[t] = __float2bfloat16(v);
  }
}

// Transpose a rows x cols BF16 matrix (row-major) into cols x rows.
__global__ void k_transpose_bf16(const __nv_bfloat16* __restrict__ in, __nv_bfloat16* __restrict__ out,
                                 int rows, int cols) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[i][threadIdx.x] = in[size_t(r) * cols + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < rows) out[size_t(c) * rows + r] = tile[threadIdx.x][i];
  }
}

__global__ void k_f32_to_bf16(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, size_t n) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    out[i] = __float2bfloat16(in[i]);
}

// Column sums of a rows x cols BF16 matrix (bias gradients), fixed order.
__global__ void k_colsum_bf16(const __nv_bfloat16* __restrict__ in, int rows, int cols, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += __bfloat162float(in[size_t(r) * cols + c]);
  out[c] = s;
}

// Probe loss and its gradient for one sample per block (Sec. 3.2.3 block S):
//   u_p = x_p - c1 J x_p + c2 J (J x_p),  r_p = u_p + O u_p - x_p,
//   loss += |r_p|^2 / (B P),  dO[r][c] = 2/(B P) sum_p r_p[r] u_p[c].
// J: n_b x n_b column-major FP32 per sample; O, dO: B rows of stride ldo >= n_b^2
// (row-major n_b x n_b block in the first n_b^2 entries); X: B x P x n_b probes.
// Dynamic shared memory: (2 P + 2) n_b floats.
__global__ void k_mlp_probe_loss(const float* __restrict__ J, const float* __restrict__ c12,
                                 const float* __restrict__ O, const float* __restrict__ X, int B, int P,
                                 int nb, int ldo, const float* __restrict__ cmean, const int* __restrict__ cls,
                                 __nv_bfloat16* __restrict__ dO, double* __restrict__ loss_part) {
  const int s = blockIdx.x;
  if (s >= B) return;
  const float* Cs = cmean + size_t(cls[s]) * ldo;   // the sample's class mean (minus I)
  extern __shared__ float sh[];
  float* su = sh;                 // P x nb
  float* sr = su + P * nb;        // P x nb
  float* sy = sr + P * nb;        // nb
  float* sz = sy + nb;            // nb
  const float* Js = J + size_t(s) * nb * nb;
  const float* Os = O + size_t(s) * ldo;
  const float c1 = c12[2 * s], c2 = c12[2 * s + 1];
  const float norm = 2.f / float(B * P);
  double lsum = 0.0;
  for (int p = 0; p < P; ++p) {
    const float* x = X + (size_t(s) * P + p) * nb;
    for (int r = threadIdx.x; r < nb; r += blockDim.x) {     // y = J x
      float a = 0.f;
      for (int c = 0; c < nb; ++c) a += Js[size_t(c) * nb + r] * x[c];
      sy[r] = a;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < nb; r += blockDim.x) {     // z = J y, u = x - c1 y + c2 z
      float a = 0.f;
      for (int c = 0; c < nb; ++c) a += Js[size_t(c) * nb + r] * sy[c];
      su[p * nb + r] = x[r] - c1 * sy[r] + c2 * a;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < nb; r += blockDim.x) {     // r_p = u + O u - x
      float a = 0.f;
      for (int c = 0; c < nb; ++c) a += (Os[size_t(r) * nb + c] + Cs[size_t(r) * nb + c]) * su[p * nb + c];
      const float rr = su[p * nb + r] + a - x[r];
      sr[p * nb + r] = rr;
      lsum += double(rr) * double(rr);
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int r = t / nb, c = t - r * nb;
    float a = 0.f;
    for (int p = 0; p < P; ++p) a += sr[p * nb + r] * su[p * nb + c];
    dO[size_t(s) * ldo + t] = __float2bfloat16(norm * a);
  }
  // block sum of the loss in a fixed order
  __shared__ double red[256];
  red[threadIdx.x] = lsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < int(blockDim.x); ++i) t += red[i];
    loss_part[s] = t / double(B * P);
  }
}

// Inverse-regression loss with the exact block inverses T = S^-1 of the BJ_ext
// path as targets (n_b x n_b column-major FP32 per sample):
//   loss = sum_s |I + O_s - T_s|_F^2 / B,   dO = 2 (I + O - T) / B,
// O, dO in the same row layout as the probe loss.
__global__ void k_mlp_inverse_loss(const float* __restrict__ T, const float* __restrict__ O, int B, int nb,
                                   int ldo, const float* __restrict__ cmean, const int* __restrict__ cls,
                                   __nv_bfloat16* __restrict__ dO, double* __restrict__ loss_part) {
  const int s = blockIdx.x;
  if (s >= B) return;
  const float* Ts = T + size_t(s) * nb * nb;
  const float* Os = O + size_t(s) * ldo;
  const float* Cs = cmean + size_t(cls[s]) * ldo;
  const float norm = 2.f / float(B);
  double lsum = 0.0;
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int r = t / nb, c = t - r * nb;
    const float d = (r == c ? 1.f : 0.f) + Os[t] + Cs[t] - Ts[size_t(c) * nb + r];
    dO[size_t(s) * ldo + t] = __float2bfloat16(norm * d);
    lsum += double(d) * double(d);
  }
  __shared__ double red[256];
  red[threadIdx.x] = lsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < int(blockDim.x); ++i) t += red[i];
    loss_part[s] = t / double(B);
  }
}

// Class means from the targets: cm[r nb + c] = mean over the samples of class
// (k1, k2) of T_i(r, c) - delta_rc, so that an untrained network already
// returns the class's mean block inverse.
__global__ void k_mlp_class_mean(const float* __restrict__ Tbuf, const float* __restrict__ cbuf, int count,
                                 int nb, float k1, float k2, float* __restrict__ cm) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nb * nb) return;
  const int r = t / nb, c = t - r * nb;
  double a = 0.0;
  int n = 0;
  for (int i = 0; i < count; ++i)
    if (cbuf[2 * i] == k1 && cbuf[2 * i + 1] == k2) { a += Tbuf[size_t(i) * nb * nb + size_t(c) * nb + r]; ++n; }
  cm[t] = n ? float(a / n) - (r == c ? 1.f : 0.f) : 0.f;
}

// Class of every sample from its (c1, c2).
__global__ void k_mlp_classify(const float* __restrict__ c12, int B, const float* __restrict__ keys,
                               int* __restrict__ cls) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < B) cls[s] = mlp_class(keys, c12[2 * s], c12[2 * s + 1]);
}

// Rademacher probes from SplitMix64 (Steele, Lea & Flood 2014) of (seed, index).
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__global__ void k_rademacher(float* __restrict__ X, size_t n, unsigned long long seed) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    X[i] = (splitmix64(seed * 0x100000001B3ull + i) >> 63) ? 1.f : -1.f;
}

// Random sample indices into the replay buffer (SplitMix64 of seed and slot).
__global__ void k_rand_idx(int* idx, int B, int count, unsigned long long seed) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < B) idx[s] = int(splitmix64(seed * 0x9E3779B97F4A7C15ull + unsigned(s)) % unsigned(count));
}

// Gather training samples (features, J, c1/c2) from the replay buffer.
__global__ void k_mlp_gather(const float* __restrict__ featbuf, const float* __restrict__ Jbuf,
                             const float* __restrict__ cbuf, const int* __restrict__ idx, int B, int din,
                             int dinp, int nb, const float* __restrict__ mu, const float* __restrict__ sd,
                             __nv_bfloat16* __restrict__ F, float* __restrict__ J, float* __restrict__ c12) {
  const int s = blockIdx.x;
  if (s >= B) return;
  const size_t src = size_t(idx[s]);
  for (int k = threadIdx.x; k < dinp; k += blockDim.x)
    F[size_t(s) * dinp + k] = __float2bfloat16(k < din ? (featbuf[src * din + k] - mu[k]) / sd[k] : 0.f);
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) J[size_t(s) * nb * nb + t] = Jbuf[src * nb * nb + t];
  if (threadIdx.x < 2) c12[2 * s + threadIdx.x] = cbuf[src * 2 + threadIdx.x];
}

// Store the features (raw, FP32), the element Jacobian (FP32) and c1, c2 of a
// set of elements into the replay buffer at rows [row0, row0 + count) (mod cap).
template <typename T>
__global__ void k_mlp_collect(const double* __restrict__ W, const T* __restrict__ Jpc, int nE, int nb,
                              double c1, double c2, int count, int stride, int offset, int row0, int cap,
                              float* __restrict__ featbuf, float* __restrict__ Jbuf, float* __restrict__ cbuf) {
  const int s = blockIdx.x;
  if (s >= count) return;
  const int e = (offset + s * stride) % nE;
  const size_t row = size_t((row0 + s) % cap);
  const int din = nb + 2;
  for (int k = threadIdx.x; k < din; k += blockDim.x) {
    float v = k < nb ? float(W[size_t(e) * nb + k]) : (k == nb ? float(c1) : float(c2));
    featbuf[row * din + k] = v;
  }
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x)
    Jbuf[row * nb * nb + t] = float(Jpc[size_t(e) * nb * nb + t]);
  if (threadIdx.x == 0) { cbuf[row * 2] = float(c1); cbuf[row * 2 + 1] = float(c2); }
}

// Store the block inverses M_e = S_e^-1 (column-major; FP64, or FP32 in the
// mixed mode) of the elements that k_mlp_collect sampled with the same (count,
// stride, offset, row0) as FP32 training targets.
template <typename T>
__global__ void k_mlp_collect_target(const T* __restrict__ Mpc, int nE, int nb, int count, int stride,
                                     int offset, int row0, int cap, float* __restrict__ Tbuf) {
  const int s = blockIdx.x;
  if (s >= count) return;
  const int e = (offset + s * stride) % nE;
  const size_t row = size_t((row0 + s) % cap);
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x)
    Tbuf[row * nb * nb + t] = float(Mpc[size_t(e) * nb * nb + t]);
}

// Adam (Kingma & Ba 2015) on FP32 parameters.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps, float bc1,
                       float bc2) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

}  // namespace hbpc
