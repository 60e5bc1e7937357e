// Internal declarations shared by the coarse-operator translation units
// (mg.cu, coarse_defl.cu); not part of the ABI.
#pragma once
#include "mg_kernels.cuh"

using dwfmg::BlockGeom;

struct dwf_coarse {
  dwf_ctx* ctx;
  BlockGeom g;
  int nb, nplus;
  double2* A64;  // [nc][9][nb][nb]
  float2* A32;   // same layout, FP32
  float* At;     // tensor-core copy (real form, TF32, K-major), built on first use
  float* At4;    // tensor-core copy (complex-split form per quad of sites), built on first use
  float* Bt;     // tensor-core right-hand sides (real form, TF32), per apply
  size_t Bt_bytes;
  int* err;      // device error flag of the tensor-core kernel (sticky)
  int* err_host; // pinned mirror, copied after every tensor-core apply
  cudaEvent_t err_ready;  // recorded after that copy
  void* ws[6];
  size_t ws_bytes[6];
  int* cg_acc;   // when set: coarse CG runs without host synchronisation and
                 // accumulates [iterations, error] here (graph capture)
  float2* Arb;   // red-black form of the operator (odd sites: A_0^-1, A_0^-1 A_d), built on first use
  // coarse deflation space (coarse_deflate): nev Ritz vectors of A^2 and 1/theta
  float2* defl_V;       // [nev][nc][nb]
  double* defl_thinv;   // device [nev]
  double2* defl_c;      // device [nev] coefficients of the current guess
  float2* defl_tmp;     // [2][nc][nb]: A r and the guess
  int defl_nev;
};

// Coarse workspace slot (grown on demand); stencil apply on CUDA cores (mg.cu).
int coarse_ws(dwf_coarse* C, int slot, size_t bytes, void** out);
int coarse_apply_dev(dwf_coarse* C, float2* out, const float2* in, int nrhs, cudaStream_t st);
// The deflation guess x0 = sum_i v_i <v_i, A r> / theta_i of the coarse CG on
// A^2 into C->defl_tmp + n (coarse_defl.cu); stream-ordered, no host sync.
int coarse_defl_guess(dwf_coarse* C, const float2* r, cudaStream_t st);
void coarse_defl_free(dwf_coarse* C);


// The coarse solves of the V-cycle on one FP32 right-hand side (mg.cu): CG on
// A^2 (from the deflation guess when a deflation space is set) and red-black
// CG on the even Schur complement squared; stream-ordered, the iteration
// count is read back unless cg_acc is set.
int coarse_cg(dwf_coarse* C, float2* e, const float2* rc, double tol, int maxiter, int* iters, cudaStream_t st);
int coarse_rb_ready(dwf_coarse* C, cudaStream_t st);
int coarse_rbcg(dwf_coarse* C, float2* e, const float2* rc, double tol, int maxiter, int* iters, cudaStream_t st);

int coarse_apply_tc(dwf_ctx* c, float2* out, const float2* in, const float2* A32, float** At, float** At4,
                    float** Bt, size_t* Bt_bytes, int nb, int nc, const int Lc[4], int nrhs, int* err_dev,
                    cudaStream_t st);
int coarse_cg_persistent(dwf_ctx* c, float2* e, const float2* rhs, const float2* A, const int Lc[4], int nc,
                         int nb, double tol, int maxiter, float2* work, double* part, int part_cap,
                         int* dev_small, int* acc, int* iters, cudaStream_t st, const float2* x0 = nullptr);
int coarse_rb_prepare(dwf_ctx* c, const double2* A64, float2* Arb, const int Lc[4], int nc, int nb, int* dev_flag,
                      cudaStream_t st);
int coarse_rbcg_persistent(dwf_ctx* c, float2* e, const float2* rhs, const float2* Arb, const int Lc[4], int nc,
                           int nb, double tol, int maxiter, float2* work, double* part, int part_cap, int* dev_small,
                           int* acc, int* iters, cudaStream_t st);

// Hybrid three-level multigrid (hybrid.cu): the levels below the fine one.
struct dwf_hybrid;
int hybrid_build(dwf_ctx* c, const dwf_mg_params* p, const dwf_hybrid_params* hp, const void* eta4, const void* eta1,
                 dwf_hybrid** out, cudaStream_t st);
void hybrid_free(dwf_hybrid* H);
// x += P1 e, e from the fixed-iteration level-1 solve of H_1 e = P1^dag r (FP32 full fields).
int hybrid_correction(dwf_hybrid* H, void* x, const void* r, cudaStream_t st, int* ncoarse);
int hybrid_level1_op(dwf_hybrid* H, int op, void* out, const void* in, int nvec, cudaStream_t st);
int hybrid_export(const dwf_hybrid* H, int what, void* out);
dwf_coarse* hybrid_coarse(dwf_hybrid* H);
double hybrid_setup_seconds(const dwf_hybrid* H);
double hybrid_coarse_seconds(const dwf_hybrid* H);
