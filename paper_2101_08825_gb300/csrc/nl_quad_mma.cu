// nl_quad_mma.cu -- nl_assemble in NL_PREC_MIXED_TF32 / NL_PREC_MIXED_BF16: the FP32 assembly
// path of nl_quad_kernel.cuh with the per-pair contraction over the outer points of Sec. 5's
// double sums (eqs. J21Nr, J22Nr) on the tensor cores (mma.sync, FP32 accumulation, two-part
// split operands).  A translation unit of its own so that these kernels compile in parallel
// with the others.
#include <cuda_runtime.h>

#include "nl_quad_kernel.cuh"

namespace nlx {

nl_status assemble_values_mma(nl_mesh* m, nl_pairs* p, const nl_kernel_params* kp,
                              const nl_quad_params* qp, nl_precision prec, double* values,
                              nl_assemble_stats* st) {
  if (prec == NL_PREC_MIXED_TF32) return assemble_single<1>(m, p, kp, qp, prec, values, st);
  if (prec == NL_PREC_MIXED_BF16) return assemble_single<2>(m, p, kp, qp, prec, values, st);
  return fail(NL_EINVAL, "nl_assemble: precision %d has no tensor-core path", (int)prec);
}

}  // namespace nlx
