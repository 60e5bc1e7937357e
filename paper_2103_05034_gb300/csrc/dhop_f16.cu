// Hopping-term and site-local fifth-dimension kernels instantiated for DWF_F16S.
#include "dhop_impl.cuh"

int dwf_launch_hop_f16(const dwfk::HopParams& hp, int Ls, int nrhs, int variant, cudaStream_t st,
                       int* nb) {
  return dwfk::launch_hop_prec<DWF_F16S>(hp, Ls, nrhs, variant, st, nb);
}

int dwf_launch_mooee_f16(void* out, const void* in, const dwfk::HopParams& hp, int dagger,
                          int inverse, int Ls, int nrhs, long long rs, cudaStream_t st) {
  return dwfk::launch_mooee_prec<DWF_F16S>(out, in, hp, dagger, inverse, Ls, nrhs, rs, st);
}
