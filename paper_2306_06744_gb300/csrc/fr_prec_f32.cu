// fr_prec_f32.cu -- instantiation of the time-step kernels with arithmetic type float.
#include "fr_kernels.cuh"

namespace frg {

int launch_traces_f32(int dim, int p, const double* u, int64_t M, const DevOps& ops, void* tr,
                     const int8_t* mask, cudaStream_t s, Err* err, const int64_t* d_M) {
  return launch_traces_impl<float>(dim, p, u, M, ops, tr, mask, s, err, d_M);
}
int launch_faces_f32(int dim, int p, FaceArgs A, const DevOps& ops, cudaStream_t s, Err* err) {
  return launch_faces_impl<float>(dim, p, A, ops, s, err);
}
int launch_stage_f32(int dim, int p, const StageArgs& A, const DevOps& ops, cudaStream_t s, Err* err) {
  return launch_stage_impl<float>(dim, p, A, ops, s, err);
}

}  // namespace frg
