// Hopping-term and site-local fifth-dimension kernels instantiated for DWF_F32.
#include "dhop_impl.cuh"

int dwf_launch_hop_f32(const dwfk::HopParams& hp, int Ls, int nrhs, int variant, cudaStream_t st,
                       int* nb) {
  return dwfk::launch_hop_prec<DWF_F32>(hp, Ls, nrhs, variant, st, nb);
}

int dwf_launch_mooee_f32(void* out, const void* in, const dwfk::HopParams& hp, int dagger,
                          int inverse, int Ls, int nrhs, long long rs, cudaStream_t st) {
  return dwfk::launch_mooee_prec<DWF_F32>(out, in, hp, dagger, inverse, Ls, nrhs, rs, st);
}
