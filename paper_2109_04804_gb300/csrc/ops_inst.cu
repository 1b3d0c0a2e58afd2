// Instantiations of the element operator kernels.  Compiled several times with
// -DHBPC_LAW, -DHBPC_DIM, -DHBPC_UNIT (a unique name) and the node-count bit masks
// -DHBPC_LOBATTO_MASK, -DHBPC_GAUSS_MASK, so that the build spreads over
// translation units compiled in parallel (see the build script).
#include "bjext.cuh"
#include "dg_ops.cuh"
#include "hbpc_internal.h"

#ifndef HBPC_LAW
#error "HBPC_LAW must be defined"
#endif
#ifndef HBPC_DIM
#error "HBPC_DIM must be defined"
#endif
#ifndef HBPC_UNIT
#error "HBPC_UNIT must be defined"
#endif

namespace hbpc {
namespace {

// cols > 1: a second grid dimension (the block columns of JobPcCols)
template <int LAW, int DIM, int P, bool LGL, class Job, typename V = double>
void launch(const Job& job, const DGParams<typename BaseOf<V>::type>& prm, cudaStream_t s, int cols = 1) {
  using KS = KernelShape<LAW, DIM, P>;
  using Gm = Geo<DIM, P>;
  constexpr size_t smem = KS::template smem_bytes<V, typename BaseOf<V>::type>();
  auto kern = &dg_operator_kernel<LAW, DIM, P, LGL, V, Job>;
  if (smem > 48 * 1024) {
    static const cudaError_t attr =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    (void)attr;
  }
  const int blocks = (prm.nE + Gm::EPB - 1) / Gm::EPB;
  kern<<<dim3(blocks, cols), Gm::THREADS, smem, s>>>(job, prm);
}

template <int LAW, int DIM, int P, bool LGL>
struct Inst {
  static constexpr int NV = KernelShape<LAW, DIM, P>::NV;
  static constexpr int NN = Geo<DIM, P>::NN;
  static constexpr bool LINEAR = LAW == LAW_ADV;

  static void r1(const DGParams<double>& p, const double* w, double* out, cudaStream_t s) {
    JobR1<NV, NN, double> j{w, out};
    launch<LAW, DIM, P, LGL>(j, p, s);
  }
  static void r2(const DGParams<double>& p, const double* w, const double* sg, double* out,
                 cudaStream_t s) {
    JobR2<NV, NN, double> j{w, sg, out};
    launch<LAW, DIM, P, LGL>(j, p, s);
  }
  static void residual(const DGParams<double>& p, const double* W, const double* S,
                       const double* b, double c1, double c2, double* G1, double* G2,
                       double* r1o, double* r2o, cudaStream_t s) {
    JobResidual<NV, NN> j{W, S, b, c1, c2, G1, G2, r1o, r2o};
    launch<LAW, DIM, P, LGL>(j, p, s);
  }
  static void jv_fd(const DGParams<double>& p, const double* W, const double* S,
                    const double* r1o, const double* r2o, const JvInput& z, const JvCoef& c,
                    cudaStream_t s) {
    JobJvFD_A<NV, NN> a{W, S, r1o, r2o, z, c};
    launch<LAW, DIM, P, LGL>(a, p, s);
    JobJvFD_B<NV, NN> b{W, S, r2o, z, c};
    launch<LAW, DIM, P, LGL>(b, p, s);
  }
  static void jv_linear(const DGParams<double>& p, const JvInput& z, const JvCoef& c,
                        cudaStream_t s) {
    if constexpr (LINEAR) {
      if (!p.visc) {   // both halves in one AdvectionPair pass
        JobJvLinearPair<NN, double, double> j{z, c};
        launch<LAW_ADV2, DIM, P, LGL>(j, p, s);
        return;
      }
    }
    JobJvLinear<NV, NN> j{z, c};
    launch<LAW, DIM, P, LGL>(j, p, s);
  }
  // mixed precision: FP32 Jacobian-vector product (Eq. 24 for a linear flux,
  // analytic dual-number form of Eq. 18 otherwise)
  static void jv_f(const DGParams<float>& p, const JvInputT<float>& z, const JvCoef& c, const float* Wf,
                   const float* Sf, cudaStream_t s) {
    if constexpr (LINEAR) {
      if (!p.visc) {
        JobJvLinearPair<NN, float, float> j{z, c};
        launch<LAW_ADV2, DIM, P, LGL, JobJvLinearPair<NN, float, float>, float>(j, p, s);
      } else {
        JobJvLinear<NV, NN, float, float> j{z, c};
        launch<LAW, DIM, P, LGL, JobJvLinear<NV, NN, float, float>, float>(j, p, s);
      }
    } else {
      JobJvMixed<NV, NN> j{Wf, Sf, z, c};
      launch<LAW, DIM, P, LGL, JobJvMixed<NV, NN>, Dual<float>>(j, p, s);
    }
  }
  // Navier-Stokes: the blocks by columns of the frozen-neighbour R2 (its
  // viscous Jacobian has no compact closed form); other laws: the analytic
  // assembly from the flux Jacobians
  static void pc_assemble(const DGParams<double>& p, const double* W, double* J, cudaStream_t s) {
    if constexpr (LAW == LAW_NS) {
      JobPcCols<NV, NN, double> j{W, J};
      launch<LAW, DIM, P, LGL, JobPcCols<NV, NN, double>, double>(j, p, s, NV * NN);
    } else {
      k_pc_assemble<LAW, DIM, P, LGL, double><<<p.nE, 128, 0, s>>>(W, J, p);
    }
  }
  // FP32 assembly for the mixed-precision mode (the blocks only precondition)
  static void pc_assemble_f(const DGParams<float>& p, const double* W, float* J, cudaStream_t s) {
    if constexpr (LAW == LAW_NS) {
      JobPcCols<NV, NN, float> j{W, J};
      launch<LAW, DIM, P, LGL, JobPcCols<NV, NN, float>, float>(j, p, s, NV * NN);
    } else {
      k_pc_assemble<LAW, DIM, P, LGL, float><<<p.nE, 128, 0, s>>>(W, J, p);
    }
  }
  // BJ^H_ext Hessian blocks (inviscid flux Hessian; no Navier-Stokes form)
  template <typename T>
  static void pc_hessian(const DGParams<T>& p, const double* W, const double* S, T* H, cudaStream_t s) {
    k_pc_assemble<LAW, DIM, P, LGL, T, true><<<p.nE, 128, 0, s>>>(W, H, p, S);
  }
  static void fill(OpsTable& t) {
    t.nv = NV;
    t.pc_assemble = &pc_assemble;
    t.pc_assemble_f = &pc_assemble_f;
    if constexpr (!LINEAR && LAW != LAW_NS) {
      t.pc_hessian = &pc_hessian<double>;
      t.pc_hessian_f = &pc_hessian<float>;
    }
    t.jv_f = &jv_f;
    t.r1 = &r1;
    t.r2 = &r2;
    t.residual = &residual;
    if constexpr (LINEAR) {
      t.jv_linear = &jv_linear;
      t.jv_fd = nullptr;
    } else {
      t.jv_fd = &jv_fd;
      t.jv_linear = nullptr;
    }
  }
};

template <bool LGL, int MASK, int P>
bool fill_if(int Preq, OpsTable& t) {
  if constexpr (((MASK >> P) & 1) != 0) {
    if (Preq == P) {
      Inst<HBPC_LAW, HBPC_DIM, P, LGL>::fill(t);
      return true;
    }
  }
  return false;
}

template <bool LGL, int MASK>
bool fill_mask(int P, OpsTable& t) {
  return fill_if<LGL, MASK, 2>(P, t) || fill_if<LGL, MASK, 3>(P, t) || fill_if<LGL, MASK, 4>(P, t) ||
         fill_if<LGL, MASK, 5>(P, t) || fill_if<LGL, MASK, 6>(P, t) || fill_if<LGL, MASK, 7>(P, t) ||
         fill_if<LGL, MASK, 8>(P, t);
}

}  // namespace

// HBPC_LOBATTO_MASK / HBPC_GAUSS_MASK: bit P set = node count P compiled in this
// unit for that node family.
#define HBPC_CAT2(a, b) a##b
#define HBPC_CAT(a, b) HBPC_CAT2(a, b)
bool HBPC_CAT(get_ops_unit_, HBPC_UNIT)(int P, bool lgl, OpsTable& t) {
  if (lgl) return fill_mask<true, HBPC_LOBATTO_MASK>(P, t);
  return fill_mask<false, HBPC_GAUSS_MASK>(P, t);
}

}  // namespace hbpc
