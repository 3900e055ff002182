// fr_prec_f64.cu -- instantiation of the time-step kernels with arithmetic type double.
#include "fr_kernels.cuh"

namespace frg {

int launch_traces_f64(int dim, int p, const double* u, int64_t M, const DevOps& ops, void* tr,
                     const int8_t* mask, cudaStream_t s, Err* err, const int64_t* d_M) {
  return launch_traces_impl<double>(dim, p, u, M, ops, tr, mask, s, err, d_M);
}
int launch_faces_f64(int dim, int p, FaceArgs A, const DevOps& ops, cudaStream_t s, Err* err) {
  return launch_faces_impl<double>(dim, p, A, ops, s, err);
}
int launch_stage_f64(int dim, int p, const StageArgs& A, const DevOps& ops, cudaStream_t s, Err* err) {
  return launch_stage_impl<double>(dim, p, A, ops, s, err);
}

}  // namespace frg
