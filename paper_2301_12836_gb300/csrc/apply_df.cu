// apply_df.cu - the forward operator in double-float arithmetic (dfloat.cuh): the kernels of
// apply.cu instantiated for dfloat in a translation unit of their own, compiled in parallel.
#define LSM_APPLY_DFLOAT_TU 1
#include "apply.cu"

namespace lsm {
template cudaError_t launch_apply<dfloat>(const Medium&, const Plans&, const ApplySys<dfloat>*, int, cudaStream_t,
                                          long long*);
}  // namespace lsm
