// Hopping-term and site-local fifth-dimension kernels instantiated for DWF_F64.
#include "dhop_impl.cuh"

int dwf_launch_hop_f64(const dwfk::HopParams& hp, int Ls, int nrhs, int variant, cudaStream_t st,
                       int* nb) {
  return dwfk::launch_hop_prec<DWF_F64>(hp, Ls, nrhs, variant, st, nb);
}

int dwf_launch_mooee_f64(void* out, const void* in, const dwfk::HopParams& hp, int dagger,
                          int inverse, int Ls, int nrhs, long long rs, cudaStream_t st) {
  return dwfk::launch_mooee_prec<DWF_F64>(out, in, hp, dagger, inverse, Ls, nrhs, rs, st);
}
