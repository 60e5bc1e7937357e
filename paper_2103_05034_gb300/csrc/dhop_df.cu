// The hopping-term kernel instantiated for FP64 storage with float-float
// arithmetic (dfloat.cuh): the FP64 operator on GB300's FP32 units.
#include "dhop_impl.cuh"
#include "dfloat.cuh"

int dwf_launch_hop_df(const dwfk::HopParams& hp, int Ls, int nrhs, int variant, cudaStream_t st, int* nb) {
  return dwfk::launch_hop_prec<DWF_P_DF>(hp, Ls, nrhs, variant, st, nb);
}
