// Wilson hopping term on every s-slice (arXiv:2103.05034, Sec. 2, Eq. 2) with
// the fifth-dimension matrix of Eq. (4) fused into the epilogue.
//
// Data layout (see include/dwfmg.h): half field [Vh][spin 4][colour 3][Ls],
// the fifth dimension innermost; links for an output parity are
// [Vh][8][3][3] with slot 2mu = U_mu(x) and slot 2mu+1 = U_mu(x-mu)^dag.
//
// Thread mapping: one CTA handles SB consecutive checkerboard sites and all
// Ls slices of each (blockDim = Ls*SB, s fastest), so
//   * the 16 (or 24) threads of one site read each spinor component of a
//     neighbour as one contiguous run of Ls complex numbers (coalesced), and
//   * the site's 8 links are loaded once into shared memory and reused by all
//     Ls threads (links cost 8*18 reals / Ls per output 5D site).
// Spin projection (1 -+ gamma_mu) reduces each neighbour to a two-spinor
// before the SU(3) multiply (chiral basis: gamma_mu = [[0,A],[A^dag,0]],
// (1 - s gamma)psi = [h; -s A^dag h], h = psi_up - s A psi_dn).
//
// Epilogue, per CTA, on the Ls-vector of every (site, spin, colour):
//   aux term   M psi_s = d psi_s - psi_{s-+1} (+ m psi at the wall), read from
//              global memory (the neighbours in s are in the same CTA's lines)
//   inverse    M_+^-1 by two O(Ls) sweeps (a forward geometric prefix sum F
//              and a backward one G, x_s = kappa/d (F_s - m G_s)), run by 12
//              threads per site on a padded shared-memory stage; M_-^-1 is the
//              same on reversed s (M_- = M_+^T, chirality - = spins 2,3)
//   Gamma_5    gamma_5 with s -> Ls-1-s on the store
//   reduction  |out|^2 in FP64 per CTA
#pragma once
#include "dwf_internal.cuh"

namespace dwfk {

struct HopParams {
  void* out;
  const void* in;
  const void* aux;
  const void* links;
  double* partials;
  int L0, L1, L2, L3, Lxh;
  int Vh;
  int zc;  // traversal z-chunk (even divisor of L2; L2 = lexicographic order)
  int l2pf; // > 0: each CTA prefetches into L2 the input rows first read by the
            // CTA l2pf positions later in the traversal (scalar kernel only)
  int out_parity;
  float sg;  // +1: D_hop, -1: D_hop^dag
  double alpha;
  int aux_mode, inv_mode, g5r5, reduce;
  long long rhs_stride;
  double d;
  // fused CG update (cg_mode = 1): with v = the operator output A p,
  // x += alpha p, r -= alpha v, |r|^2 reduced; v itself is not stored.
  int cg_mode;
  void* cg_x;
  void* cg_r;
  const void* cg_p;
  const double* cg_alpha;  // device scalars, cg_alpha[rhs * cg_astride]
  int cg_astride;          // 0: one alpha for every rhs
  int cg_x32;              // x stored in FP32 (with FP16-storage r and p)
  // fused Chebyshev recurrence step (cheb_mode = 1) instead of storing the
  // operator output v (after the Gamma_5 store mapping):
  //   tp = ta v + tb x - tp;  acc += cacc tp (acc may be null)
  int cheb_mode;
  const void* cheb_x;
  void* cheb_tp;
  void* cheb_acc;
  double cheb_ta, cheb_tb, cheb_cacc;
  double m[DWF_MAX_RHS];
  double kappa[DWF_MAX_RHS];
  double dls1[DWF_MAX_RHS];
};

template <class R>
__device__ __forceinline__ void cacc(cpx<R>& a, const cpx<R>& b) {
  a.re += b.re;
  a.im += b.im;
}

// Products with the hopping sign sg = +-1 (overloaded for arithmetic types
// in which a product costs more than a sign change).
template <class R>
__device__ __forceinline__ R sg_mul(R sg, R x) {
  return sg * x;
}
template <class R>
__device__ __forceinline__ R sg_fma(R sg, R x, R y) {
  return fma(sg, x, y);
}

// acc += (1 - sg gamma_mu) U psi, spin-projected.
template <class R, int MU>
__device__ __forceinline__ void hop_dir(cpx<R> (&acc)[12], const cpx<R> (&ps)[12],
                                        const cpx<R>* __restrict__ U, R sg) {
  cpx<R> h0[3], h1[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const cpx<R> p0 = ps[c], p1 = ps[3 + c], p2 = ps[6 + c], p3 = ps[9 + c];
    if (MU == 0) {  // A = -i sigma_1: h0 = p0 + s i p3, h1 = p1 + s i p2
      h0[c] = cmake<R>(p0.re - sg_mul(sg, p3.im), p0.im + sg_mul(sg, p3.re));
      h1[c] = cmake<R>(p1.re - sg_mul(sg, p2.im), p1.im + sg_mul(sg, p2.re));
    } else if (MU == 1) {  // A = -i sigma_2: h0 = p0 + s p3, h1 = p1 - s p2
      h0[c] = cmake<R>(p0.re + sg_mul(sg, p3.re), p0.im + sg_mul(sg, p3.im));
      h1[c] = cmake<R>(p1.re - sg_mul(sg, p2.re), p1.im - sg_mul(sg, p2.im));
    } else if (MU == 2) {  // A = -i sigma_3: h0 = p0 + s i p2, h1 = p1 - s i p3
      h0[c] = cmake<R>(p0.re - sg_mul(sg, p2.im), p0.im + sg_mul(sg, p2.re));
      h1[c] = cmake<R>(p1.re + sg_mul(sg, p3.im), p1.im - sg_mul(sg, p3.re));
    } else {  // A = 1: h0 = p0 - s p2, h1 = p1 - s p3
      h0[c] = cmake<R>(p0.re - sg_mul(sg, p2.re), p0.im - sg_mul(sg, p2.im));
      h1[c] = cmake<R>(p1.re - sg_mul(sg, p3.re), p1.im - sg_mul(sg, p3.im));
    }
  }
#pragma unroll
  for (int a = 0; a < 3; a++) {
    cpx<R> g0 = cmake<R>(0, 0), g1 = cmake<R>(0, 0);
#pragma unroll
    for (int b = 0; b < 3; b++) {
      const cpx<R> u = U[a * 3 + b];
      g0.re = fma(u.re, h0[b].re, g0.re);
      g0.re = fma(-u.im, h0[b].im, g0.re);
      g0.im = fma(u.re, h0[b].im, g0.im);
      g0.im = fma(u.im, h0[b].re, g0.im);
      g1.re = fma(u.re, h1[b].re, g1.re);
      g1.re = fma(-u.im, h1[b].im, g1.re);
      g1.im = fma(u.re, h1[b].im, g1.im);
      g1.im = fma(u.im, h1[b].re, g1.im);
    }
    cacc(acc[a], g0);
    cacc(acc[3 + a], g1);
    // lower spins: -s A^dag g
    if (MU == 0) {  // A^dag g = (i g1, i g0)
      acc[6 + a].re = sg_fma(sg, g1.im, acc[6 + a].re);
      acc[6 + a].im = sg_fma(-sg, g1.re, acc[6 + a].im);
      acc[9 + a].re = sg_fma(sg, g0.im, acc[9 + a].re);
      acc[9 + a].im = sg_fma(-sg, g0.re, acc[9 + a].im);
    } else if (MU == 1) {  // A^dag g = (g1, -g0)
      acc[6 + a].re = sg_fma(-sg, g1.re, acc[6 + a].re);
      acc[6 + a].im = sg_fma(-sg, g1.im, acc[6 + a].im);
      acc[9 + a].re = sg_fma(sg, g0.re, acc[9 + a].re);
      acc[9 + a].im = sg_fma(sg, g0.im, acc[9 + a].im);
    } else if (MU == 2) {  // A^dag g = (i g0, -i g1)
      acc[6 + a].re = sg_fma(sg, g0.im, acc[6 + a].re);
      acc[6 + a].im = sg_fma(-sg, g0.re, acc[6 + a].im);
      acc[9 + a].re = sg_fma(-sg, g1.im, acc[9 + a].re);
      acc[9 + a].im = sg_fma(sg, g1.re, acc[9 + a].im);
    } else {  // A^dag g = (g0, g1)
      acc[6 + a].re = sg_fma(-sg, g0.re, acc[6 + a].re);
      acc[6 + a].im = sg_fma(-sg, g0.im, acc[6 + a].im);
      acc[9 + a].re = sg_fma(-sg, g1.re, acc[9 + a].re);
      acc[9 + a].im = sg_fma(-sg, g1.im, acc[9 + a].im);
    }
  }
}

// ---------------------------------------------------------------- packed FP32
// sm_100+ executes fma/add on a pair of FP32 values held in one 64-bit
// register (fma.rn.f32x2).  A complex number (re, im) is one such pair, so a
// complex multiply-add takes two packed FMAs: (u_re, u_re)*(h_re, h_im) +
// (-u_im, u_im)*(h_im, h_re).  Links are staged in shared memory already
// broadcast as (re, re, -im, im).
typedef unsigned long long f2p;
__device__ __forceinline__ f2p pk2(float a, float b) {
  f2p r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk2(f2p v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2p fma2(f2p a, f2p b, f2p c) {
  f2p d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2p add2(f2p a, f2p b) {
  f2p d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2p swp2(f2p a) {
  float x, y;
  upk2(a, x, y);
  return pk2(y, x);
}

// acc += (1 - sg gamma_mu) U psi with packed arithmetic; sgp = (sg, sg),
// sgv = (-sg, sg) (multiplication by sg*i of a swapped pair).
template <int MU>
__device__ __forceinline__ void hop_dir_x2(f2p (&acc)[12], const f2p (&ps)[12], const float4* __restrict__ U,
                                           f2p sgp, f2p sgv, f2p nsgp, f2p nsgv) {
  f2p h0[3], h1[3], s0[3], s1[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const f2p p0 = ps[c], p1 = ps[3 + c], p2 = ps[6 + c], p3 = ps[9 + c];
    if (MU == 0) {  // h0 = p0 + s i p3, h1 = p1 + s i p2
      h0[c] = fma2(sgv, swp2(p3), p0);
      h1[c] = fma2(sgv, swp2(p2), p1);
    } else if (MU == 1) {  // h0 = p0 + s p3, h1 = p1 - s p2
      h0[c] = fma2(sgp, p3, p0);
      h1[c] = fma2(nsgp, p2, p1);
    } else if (MU == 2) {  // h0 = p0 + s i p2, h1 = p1 - s i p3
      h0[c] = fma2(sgv, swp2(p2), p0);
      h1[c] = fma2(nsgv, swp2(p3), p1);
    } else {  // h0 = p0 - s p2, h1 = p1 - s p3
      h0[c] = fma2(nsgp, p2, p0);
      h1[c] = fma2(nsgp, p3, p1);
    }
    s0[c] = swp2(h0[c]);
    s1[c] = swp2(h1[c]);
  }
#pragma unroll
  for (int a = 0; a < 3; a++) {
    f2p g0 = 0ull, g1 = 0ull;  // +0.0f pairs
#pragma unroll
    for (int b = 0; b < 3; b++) {
      const float4 u = U[a * 3 + b];
      const f2p ure = pk2(u.x, u.y), uim = pk2(u.z, u.w);
      g0 = fma2(ure, h0[b], g0);
      g0 = fma2(uim, s0[b], g0);
      g1 = fma2(ure, h1[b], g1);
      g1 = fma2(uim, s1[b], g1);
    }
    acc[a] = add2(acc[a], g0);
    acc[3 + a] = add2(acc[3 + a], g1);
    if (MU == 0) {  // lower: -s i g1, -s i g0
      acc[6 + a] = fma2(nsgv, swp2(g1), acc[6 + a]);
      acc[9 + a] = fma2(nsgv, swp2(g0), acc[9 + a]);
    } else if (MU == 1) {  // -s g1, s g0
      acc[6 + a] = fma2(nsgp, g1, acc[6 + a]);
      acc[9 + a] = fma2(sgp, g0, acc[9 + a]);
    } else if (MU == 2) {  // -s i g0, s i g1
      acc[6 + a] = fma2(nsgv, swp2(g0), acc[6 + a]);
      acc[9 + a] = fma2(sgv, swp2(g1), acc[9 + a]);
    } else {  // -s g0, -s g1
      acc[6 + a] = fma2(nsgp, g0, acc[6 + a]);
      acc[9 + a] = fma2(nsgp, g1, acc[9 + a]);
    }
  }
}

template <int P, int LS>
__device__ __forceinline__ void load_spinor_x2(f2p (&ps)[12], const typename Prec<P>::S* __restrict__ base) {
#pragma unroll
  for (int c = 0; c < 12; c++) {
    const auto z = ld_c(base + c * LS);
    ps[c] = pk2((float)z.re, (float)z.im);
  }
}

template <int P, int LS>
__device__ __forceinline__ void load_spinor(cpx<typename Prec<P>::R> (&ps)[12],
                                            const typename Prec<P>::S* __restrict__ base, int s) {
#pragma unroll
  for (int c = 0; c < 12; c++) ps[c] = ld_c(base + c * LS + s);
}

// M_+^-1 (fwd=true) or M_-^-1 (fwd=false, reversed s) of one Ls-row, in place.
template <class R, int LS>
__device__ __forceinline__ void minv_row(cpx<R>* row, bool fwd, R d, R m, R kappa, R dls1) {
  cpx<R> val[LS], G[LS];
#pragma unroll
  for (int q = 0; q < LS; q++) val[q] = row[fwd ? q : LS - 1 - q];
  cpx<R> g = cmake<R>(0, 0);
#pragma unroll
  for (int q = LS - 1; q >= 0; q--) {
    G[q] = g;
    g.re = fma(d, g.re, dls1 * val[q].re);
    g.im = fma(d, g.im, dls1 * val[q].im);
  }
  const R dinv = R(1) / d;
  const R kd = kappa * dinv;
  cpx<R> f = cmake<R>(0, 0);
#pragma unroll
  for (int q = 0; q < LS; q++) {
    f.re = fma(f.re, dinv, val[q].re);
    f.im = fma(f.im, dinv, val[q].im);
    cpx<R> o;
    o.re = kd * fma(-m, G[q].re, f.re);
    o.im = kd * fma(-m, G[q].im, f.im);
    row[fwd ? q : LS - 1 - q] = o;
  }
}

// The same inverse in place with O(1) registers (shared-memory rows): a
// forward pass leaves F_q in the row, the backward pass recovers
// v_q = F_q - F_{q-1}/d, accumulates G and writes x_q = kappa/d (F_q - m G_q).
template <class R, int LS>
__device__ __forceinline__ void minv_row_inplace(cpx<R>* row, bool fwd, R d, R m, R kappa, R dls1) {
  const R dinv = R(1) / d;
  const R kd = kappa * dinv;
  cpx<R> f = cmake<R>(0, 0);
#pragma unroll 4
  for (int q = 0; q < LS; q++) {
    cpx<R>& e = row[fwd ? q : LS - 1 - q];
    f.re = fma(f.re, dinv, e.re);
    f.im = fma(f.im, dinv, e.im);
    e = f;
  }
  cpx<R> g = cmake<R>(0, 0);
  cpx<R> Fq = row[fwd ? LS - 1 : 0];
#pragma unroll 4
  for (int q = LS - 1; q >= 0; q--) {
    const cpx<R> Fm = q > 0 ? row[fwd ? q - 1 : LS - q] : cmake<R>(0, 0);
    const cpx<R> vq = cmake<R>(fma(-dinv, Fm.re, Fq.re), fma(-dinv, Fm.im, Fq.im));
    row[fwd ? q : LS - 1 - q] = cmake<R>(kd * fma(-m, g.re, Fq.re), kd * fma(-m, g.im, Fq.im));
    g.re = fma(d, g.re, dls1 * vq.re);
    g.im = fma(d, g.im, dls1 * vq.im);
    Fq = Fm;
  }
}

extern __shared__ __align__(16) unsigned char hop_dyn_smem[];

// Bulk prefetch of [p, p + bytes) into L2 (p and bytes multiples of 16).
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Register cap: REGS registers per thread give at least 65536/(LS*SB*REGS)
// resident CTAs per SM (REGS = 0: no cap).  PF: prefetch the next neighbour.
template <int LS, int SB, int REGS>
struct HopMinBlocks {
  static constexpr int v = REGS == 0 ? 1 : (65536 / (LS * SB * REGS) > 0 ? 65536 / (LS * SB * REGS) : 1);
};

// RY > 1: the CTA covers RY consecutive y-rows of SB sites each (same x
// segment), so a row's +-y neighbours and the next row's +-x neighbours are
// the same input sites and are shared through L1.
template <int P, int LS, int SB, int REGS, int PF, int RY = 1>
__global__ void __launch_bounds__(LS* SB* RY, (HopMinBlocks<LS, SB * RY, REGS>::v)) hop_kernel(const HopParams p) {
  typedef typename Prec<P>::S S;
  typedef typename Prec<P>::R R;
  typedef typename Prec<P>::LS LT;
  constexpr int SBC = SB * RY;  // sites per CTA
  constexpr int NT = LS * SBC;
  // PF == 2 (packed FP32 arithmetic) keeps each link element as (re, re, -im, im)
  // dynamic shared memory: the links during the hop, then (inv_mode only)
  // the M_ee^-1 stage in the same bytes; the launcher sizes it per launch so
  // that plain hops leave most of the SM's L1 to the neighbour re-reads
  cpx<R>* sU = (cpx<R>*)hop_dyn_smem;
  cpx<R>* stage = (cpx<R>*)hop_dyn_smem;
  __shared__ double red[NT / 32 + 1];

  const int tid = threadIdx.x;
  const int sl = tid / LS;
  const int s = tid - sl * LS;
  // Traversal order: CTAs walk z-chunks of zc planes outermost and t inside
  // them, so the t +- 1 neighbour slices of the chunk stay resident in L2 on
  // lattices whose full time slice does not fit (zc = L2 is the plain
  // lexicographic order).
  const int zc = p.zc;
  const int rhs = blockIdx.y;
  auto cta_site0 = [&](int bx) -> int {
    if (RY > 1 || (!(PF == 3) && zc < p.L2 && (p.Lxh % SB) == 0)) {
      // (RY > 1 needs SB | Lxh and RY | L1; the host launches it only then)
      const int nseg = p.Lxh / SB;
      const int ny = p.L1 / RY;
      int r = bx;
      const int seg = r % nseg;
      r /= nseg;
      const int yy = (r % ny) * RY;
      r /= ny;
      const int zl = r % zc;
      r /= zc;
      const int tt = r % p.L3;
      const int zz = (r / p.L3) * zc + zl;
      return ((tt * p.L2 + zz) * p.L1 + yy) * p.Lxh + seg * SB;
    }
    return bx * SB;
  };
  const int site0 = cta_site0(blockIdx.x);
  if (PF == 0 && RY == 1 && p.l2pf > 0 && tid == 0 && blockIdx.x + p.l2pf < gridDim.x) {
    // The rows a CTA reads first in the traversal are the t+1 and z+1
    // neighbour rows of its own row; fetch those of a CTA that starts about a
    // wave later into L2 now, so that its first reads hit L2.
    const int s2 = cta_site0(blockIdx.x + p.l2pf);  // < Vh: the CTA exists
    int rr = s2 / p.Lxh;
    const int y2 = rr % p.L1;
    rr /= p.L1;
    const int z2 = rr % p.L2;
    const int t2 = rr / p.L2;
    const int zq = z2 + 1 == p.L2 ? 0 : z2 + 1, tq = t2 + 1 == p.L3 ? 0 : t2 + 1;
    const unsigned rowb = (unsigned)(p.Lxh * 12 * LS * sizeof(S));
    const char* base = (const char*)((const S*)p.in + (size_t)rhs * p.rhs_stride);
    if ((((uintptr_t)base) & 15) == 0 && (rowb & 15) == 0) {  // bulk-copy alignment
      prefetch_l2(base + (size_t)((tq * p.L2 + z2) * p.L1 + y2) * rowb, rowb);
      prefetch_l2(base + (size_t)((t2 * p.L2 + zq) * p.L1 + y2) * rowb, rowb);
    }
  }
  // site of the l-th CTA slot (rows of SB sites, Lxh apart)
  auto row_site = [&](int l) { return RY > 1 ? site0 + (l / SB) * p.Lxh + (l % SB) : site0 + l; };
  // PF == 3: the CTA handles the 8 output-parity sites of one 2^4 hypercube
  // (SB = 8), so half of every site's neighbours are the hypercube's other 8
  // sites, shared through L1 by the CTA.  Otherwise SB consecutive sites.
  constexpr bool TILE = (PF == 3);
  auto tile_coords = [&](int l, int& X, int& Y, int& Z, int& T) {
    // corners (dx dy dz dt as bits 3..0) of each parity, in a fixed order
    const int even_c[8] = {0x0, 0xC, 0xA, 0x9, 0x6, 0x5, 0x3, 0xF};
    const int odd_c[8] = {0x8, 0x4, 0x2, 0x1, 0xE, 0xD, 0xB, 0x7};
    const int code = p.out_parity ? odd_c[l] : even_c[l];
    const int hx = p.L0 >> 1, hy = p.L1 >> 1, hz = p.L2 >> 1, ht = p.L3 >> 1, zc2 = p.zc >> 1;
    int r = blockIdx.x;
    const int cx = r % hx;
    r /= hx;
    const int cy = r % hy;
    r /= hy;
    int cz, ct;
    if (zc2 > 0 && zc2 < hz) {  // z-chunked hypercube order
      const int czl = r % zc2;
      r /= zc2;
      ct = r % ht;
      cz = (r / ht) * zc2 + czl;
    } else {
      cz = r % hz;
      ct = r / hz;
    }
    X = 2 * cx + ((code >> 3) & 1);
    Y = 2 * cy + ((code >> 2) & 1);
    Z = 2 * cz + ((code >> 1) & 1);
    T = 2 * ct + (code & 1);
  };
  auto tile_site = [&](int l) {
    int X, Y, Z, T;
    tile_coords(l, X, Y, Z, T);
    return ((T * p.L2 + Z) * p.L1 + Y) * p.Lxh + (X >> 1);
  };
  const int site = TILE ? tile_site(sl) : row_site(sl);
  const bool active = site < p.Vh;

  // coordinates and the first neighbour's spinor are fetched before the
  // link barrier, so that the two latencies overlap (inactive threads of a
  // ragged last CTA compute addresses of site 0 and load nothing)
  int x, y, z, t;
  if (TILE) {
    tile_coords(sl, x, y, z, t);
  } else {
    int rem = (active ? site : 0) / p.Lxh;
    const int xh = (active ? site : 0) - rem * p.Lxh;
    y = rem % p.L1;
    rem /= p.L1;
    z = rem % p.L2;
    t = rem / p.L2;
    x = 2 * xh + ((y + z + t + p.out_parity) & 1);
  }
  const S* in = (const S*)p.in + (size_t)rhs * p.rhs_stride;
  const int Lxh = p.Lxh, L1 = p.L1, L2 = p.L2;
  auto cbi = [&](int X, int Y, int Z, int T) { return ((T * L2 + Z) * L1 + Y) * Lxh + (X >> 1); };
  const int xp = (x + 1 == p.L0) ? 0 : x + 1, xm = (x == 0) ? p.L0 - 1 : x - 1;
  const int yp = (y + 1 == p.L1) ? 0 : y + 1, ym = (y == 0) ? p.L1 - 1 : y - 1;
  const int zp = (z + 1 == p.L2) ? 0 : z + 1, zm = (z == 0) ? p.L2 - 1 : z - 1;
  const int tp = (t + 1 == p.L3) ? 0 : t + 1, tm = (t == 0) ? p.L3 - 1 : t - 1;
  const R sf = (R)p.sg;
  const cpx<R>* U = sU + sl * 72;
  in += s;
  auto nbp = [&](int d) -> const S* {
    int X = x, Y = y, Z = z, T = t;
    switch (d) {
      case 0: X = xp; break;
      case 1: X = xm; break;
      case 2: Y = yp; break;
      case 3: Y = ym; break;
      case 4: Z = zp; break;
      case 5: Z = zm; break;
      case 6: T = tp; break;
      default: T = tm; break;
    }
    return in + (size_t)cbi(X, Y, Z, T) * (12 * LS);
  };
  cpx<R> ps[12];
  if ((PF == 0 || PF == 3) && active) load_spinor<P, LS>(ps, nbp(0), 0);  // the scalar paths
  {
    const LT* gl = (const LT*)p.links + (size_t)site0 * 72;
    const int n = (TILE || RY > 1) ? SBC * 72 : min(SB, p.Vh - site0) * 72;
    for (int i = tid; i < n; i += NT) {
      const LT v = TILE     ? ((const LT*)p.links)[(size_t)tile_site(i / 72) * 72 + (i % 72)]
                   : RY > 1 ? ((const LT*)p.links)[(size_t)row_site(i / 72) * 72 + (i % 72)]
                            : gl[i];
      if constexpr (PF == 2) {
        ((float4*)sU)[i] = make_float4((float)v.x, (float)v.x, -(float)v.y, (float)v.y);
      } else {
        sU[i] = cmake<R>((R)v.x, (R)v.y);
      }
    }
  }
  __syncthreads();

  cpx<R> v[12];
#pragma unroll
  for (int c = 0; c < 12; c++) v[c] = cmake<R>(0, 0);

  if (active) {
    if constexpr (PF == 2) {
      const float4* U4 = (const float4*)sU + sl * 72;
      const float sgf = (float)p.sg;
      const f2p sgp = pk2(sgf, sgf), nsgp = pk2(-sgf, -sgf), sgv = pk2(-sgf, sgf), nsgv = pk2(sgf, -sgf);
      f2p acc[12], pq[12];
#pragma unroll
      for (int c = 0; c < 12; c++) acc[c] = 0ull;
      load_spinor_x2<P, LS>(pq, nbp(0));
      hop_dir_x2<0>(acc, pq, U4 + 0 * 9, sgp, sgv, nsgp, nsgv);
      load_spinor_x2<P, LS>(pq, nbp(1));
      hop_dir_x2<0>(acc, pq, U4 + 1 * 9, nsgp, nsgv, sgp, sgv);
      load_spinor_x2<P, LS>(pq, nbp(2));
      hop_dir_x2<1>(acc, pq, U4 + 2 * 9, sgp, sgv, nsgp, nsgv);
      load_spinor_x2<P, LS>(pq, nbp(3));
      hop_dir_x2<1>(acc, pq, U4 + 3 * 9, nsgp, nsgv, sgp, sgv);
      load_spinor_x2<P, LS>(pq, nbp(4));
      hop_dir_x2<2>(acc, pq, U4 + 4 * 9, sgp, sgv, nsgp, nsgv);
      load_spinor_x2<P, LS>(pq, nbp(5));
      hop_dir_x2<2>(acc, pq, U4 + 5 * 9, nsgp, nsgv, sgp, sgv);
      load_spinor_x2<P, LS>(pq, nbp(6));
      hop_dir_x2<3>(acc, pq, U4 + 6 * 9, sgp, sgv, nsgp, nsgv);
      load_spinor_x2<P, LS>(pq, nbp(7));
      hop_dir_x2<3>(acc, pq, U4 + 7 * 9, nsgp, nsgv, sgp, sgv);
#pragma unroll
      for (int c = 0; c < 12; c++) {
        float a, b;
        upk2(acc[c], a, b);
        v[c] = cmake<R>((R)a, (R)b);
      }
    } else if (PF == 1) {
      // register double buffer: the loads of neighbour d+1 are in flight while
      // neighbour d is projected and multiplied
      cpx<R> pa[12], pb[12];
      load_spinor<P, LS>(pa, nbp(0), 0);
      load_spinor<P, LS>(pb, nbp(1), 0);
      hop_dir<R, 0>(v, pa, U + 0 * 9, sf);
      load_spinor<P, LS>(pa, nbp(2), 0);
      hop_dir<R, 0>(v, pb, U + 1 * 9, -sf);
      load_spinor<P, LS>(pb, nbp(3), 0);
      hop_dir<R, 1>(v, pa, U + 2 * 9, sf);
      load_spinor<P, LS>(pa, nbp(4), 0);
      hop_dir<R, 1>(v, pb, U + 3 * 9, -sf);
      load_spinor<P, LS>(pb, nbp(5), 0);
      hop_dir<R, 2>(v, pa, U + 4 * 9, sf);
      load_spinor<P, LS>(pa, nbp(6), 0);
      hop_dir<R, 2>(v, pb, U + 5 * 9, -sf);
      load_spinor<P, LS>(pb, nbp(7), 0);
      hop_dir<R, 3>(v, pa, U + 6 * 9, sf);
      hop_dir<R, 3>(v, pb, U + 7 * 9, -sf);
    } else {
      hop_dir<R, 0>(v, ps, U + 0 * 9, sf);  // ps holds neighbour 0 already
      load_spinor<P, LS>(ps, nbp(1), 0);
      hop_dir<R, 0>(v, ps, U + 1 * 9, -sf);
      load_spinor<P, LS>(ps, nbp(2), 0);
      hop_dir<R, 1>(v, ps, U + 2 * 9, sf);
      load_spinor<P, LS>(ps, nbp(3), 0);
      hop_dir<R, 1>(v, ps, U + 3 * 9, -sf);
      load_spinor<P, LS>(ps, nbp(4), 0);
      hop_dir<R, 2>(v, ps, U + 4 * 9, sf);
      load_spinor<P, LS>(ps, nbp(5), 0);
      hop_dir<R, 2>(v, ps, U + 5 * 9, -sf);
      load_spinor<P, LS>(ps, nbp(6), 0);
      hop_dir<R, 3>(v, ps, U + 6 * 9, sf);
      load_spinor<P, LS>(ps, nbp(7), 0);
      hop_dir<R, 3>(v, ps, U + 7 * 9, -sf);
    }

    const R alpha = (R)p.alpha;
#pragma unroll
    for (int c = 0; c < 12; c++) {
      v[c].re *= alpha;
      v[c].im *= alpha;
    }
    if (p.aux_mode) {
      const S* aux = (const S*)p.aux + (size_t)rhs * p.rhs_stride + (size_t)site * 12 * LS;
      if (p.aux_mode == 1) {
#pragma unroll
        for (int c = 0; c < 12; c++) cacc(v[c], ld_c(aux + c * LS + s));
      } else {
        const bool dagM = p.aux_mode == 3;
        const R d = (R)p.d, m = (R)p.m[rhs];
        // chirality + (spins 0,1) non-dagger: M_+ couples s-1; chirality -: s+1
        const int sm = s > 0 ? s - 1 : LS - 1;
        const int sp = s < LS - 1 ? s + 1 : 0;
        const R cm = s > 0 ? R(-1) : m;
        const R cp = s < LS - 1 ? R(-1) : m;
#pragma unroll
        for (int c = 0; c < 12; c++) {
          const bool lower = (c < 6) != dagM;
          const cpx<R> a = ld_c(aux + c * LS + s);
          const cpx<R> an = ld_c(aux + c * LS + (lower ? sm : sp));
          const R co = lower ? cm : cp;
          v[c].re += fma(d, a.re, co * an.re);
          v[c].im += fma(d, a.im, co * an.im);
        }
      }
    }
  }

  if (p.inv_mode) {
    __syncthreads();  // every thread is done with the links
    if (active) {
#pragma unroll
      for (int c = 0; c < 12; c++) stage[(sl * 12 + c) * (LS + 1) + s] = v[c];
    }
    __syncthreads();
    for (int w = tid; w < SBC * 12; w += NT) {
      const int sl2 = w / 12, c2 = w - sl2 * 12;
      if ((TILE || RY > 1) || site0 + sl2 < p.Vh) {
        const bool fwd = (c2 < 6) != (p.inv_mode == 2);
        minv_row_inplace<R, LS>(stage + (sl2 * 12 + c2) * (LS + 1), fwd, (R)p.d, (R)p.m[rhs],
                        (R)p.kappa[rhs], (R)p.dls1[rhs]);
      }
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int c = 0; c < 12; c++) v[c] = stage[(sl * 12 + c) * (LS + 1) + s];
    }
  }

  if (p.cg_mode) {
    // CG update on the operator output v = A p: x += alpha p, r -= alpha v;
    // v becomes the new residual for the reduction below
    if (active) {
      const size_t off = (size_t)rhs * p.rhs_stride + (size_t)site * 12 * LS + s;
      S* xs = (S*)p.cg_x + off;
      float2* xs32 = (float2*)p.cg_x + off;
      S* rs = (S*)p.cg_r + off;
      const S* ps = (const S*)p.cg_p + off;
      const R alpha = (R)p.cg_alpha[(size_t)rhs * p.cg_astride];
      const bool x32 = (P == DWF_F16S) && p.cg_x32;
#pragma unroll
      for (int c = 0; c < 12; c++) {
        cpx<R> xv, rv = ld_c(rs + c * LS);
        if (x32) {
          const float2 t = xs32[c * LS];
          xv = cmake<R>((R)t.x, (R)t.y);
        } else {
          xv = ld_c(xs + c * LS);
        }
        const cpx<R> pv = ld_c(ps + c * LS);
        xv.re = fma(alpha, pv.re, xv.re);
        xv.im = fma(alpha, pv.im, xv.im);
        rv.re = fma(-alpha, v[c].re, rv.re);
        rv.im = fma(-alpha, v[c].im, rv.im);
        if (x32)
          xs32[c * LS] = make_float2((float)xv.re, (float)xv.im);
        else
          st_c(xs + c * LS, xv);
        st_c(rs + c * LS, rv);
        v[c] = rv;
      }
    }
  } else if (active && p.cheb_mode) {
    const size_t base = (size_t)rhs * p.rhs_stride + (size_t)site * 12 * LS;
    const int so = p.g5r5 ? LS - 1 - s : s;
    const S* cx = (const S*)p.cheb_x + base;
    S* ct = (S*)p.cheb_tp + base;
    S* ca = p.cheb_acc ? (S*)p.cheb_acc + base : nullptr;
    const R ta = (R)p.cheb_ta, tb = (R)p.cheb_tb, cc = (R)p.cheb_cacc;
#pragma unroll
    for (int c = 0; c < 12; c++) {
      cpx<R> o = v[c];
      if (p.g5r5 && c >= 6) {
        o.re = -o.re;
        o.im = -o.im;
      }
      const cpx<R> xv = ld_c(cx + c * LS + so), tv = ld_c(ct + c * LS + so);
      cpx<R> w;
      w.re = fma(ta, o.re, fma(tb, xv.re, -tv.re));
      w.im = fma(ta, o.im, fma(tb, xv.im, -tv.im));
      st_c(ct + c * LS + so, w);
      if (ca) {
        cpx<R> av = ld_c(ca + c * LS + so);
        av.re = fma(cc, w.re, av.re);
        av.im = fma(cc, w.im, av.im);
        st_c(ca + c * LS + so, av);
      }
    }
  } else if (active) {
    S* out = (S*)p.out + (size_t)rhs * p.rhs_stride + (size_t)site * 12 * LS;
    if (p.g5r5) {
      const int so = LS - 1 - s;
#pragma unroll
      for (int c = 0; c < 12; c++) {
        cpx<R> o = v[c];
        if (c >= 6) {
          o.re = -o.re;
          o.im = -o.im;
        }
        st_c(out + c * LS + so, o);
      }
    } else {
#pragma unroll
      for (int c = 0; c < 12; c++) st_c(out + c * LS + s, v[c]);
    }
  }

  if (p.reduce) {
    PartialSum<R> ps;
    if (active) {
#pragma unroll
      for (int c = 0; c < 12; c++) ps.add(fma(v[c].re, v[c].re, v[c].im * v[c].im));
    }
    double acc = ps.value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();
    if (tid == 0) {
      double tot = 0.0;
      for (int i = 0; i < NT / 32; i++) tot += red[i];
      p.partials[blockIdx.y * gridDim.x + blockIdx.x] = tot;
    }
  }
}

// Rows of Ls complex numbers per CTA of the site-local kernel: 128, or 64
// where 128 padded rows would exceed 48 KB of static shared memory.
template <int P, int LS>
struct MooRows {
  static constexpr int v =
      128 * (LS + 1) * sizeof(cpx<typename Prec<P>::R>) <= 48 * 1024 ? 128 : 64;
};

// Site-local M, M^dag, M^-1 or M^-dag of Eq. (4) on whole Ls-rows, one row
// (site, spin, colour) per thread.  The CTA's rows are moved between global
// and shared memory with consecutive threads on consecutive numbers, so that
// the global accesses are coalesced; each thread works on its own row in
// registers.
template <int P, int LS>
__global__ void __launch_bounds__(128) mooee_kernel(typename Prec<P>::S* out,
                                                    const typename Prec<P>::S* in, int Vh,
                                                    int dagger, int inverse, long long rhs_stride,
                                                    HopParams p) {
  typedef typename Prec<P>::R R;
  typedef typename Prec<P>::S S;
  constexpr int RB = MooRows<P, LS>::v;
  __shared__ cpx<R> tile[RB * (LS + 1)];
  const int tid = threadIdx.x;
  const int rhs = blockIdx.y;
  const long long nrows = (long long)Vh * 12;
  const long long row0 = (long long)blockIdx.x * RB;
  const int nr = (int)(nrows - row0 < RB ? nrows - row0 : RB);
  const size_t base = (size_t)rhs * rhs_stride + (size_t)row0 * LS;
  const S* src = in + base;
  for (int e = tid; e < nr * LS; e += 128) {
    const int r = e / LS, q = e - r * LS;
    tile[r * (LS + 1) + q] = ld_c(src + e);
  }
  __syncthreads();
  if (tid < nr) {
    cpx<R>* rp = tile + tid * (LS + 1);
    const int c = (int)((row0 + tid) % 12);
    cpx<R> row[LS];
#pragma unroll
    for (int q = 0; q < LS; q++) row[q] = rp[q];
    const R d = (R)p.d, m = (R)p.m[rhs];
    const bool plus_rule = (c < 6) != (dagger != 0);  // M_+ type (couples s-1)
    if (inverse) {
      minv_row<R, LS>(row, plus_rule, d, m, (R)p.kappa[rhs], (R)p.dls1[rhs]);
    } else {
      cpx<R> res[LS];
#pragma unroll
      for (int q = 0; q < LS; q++) {
        int qn;
        R co;
        if (plus_rule) {
          qn = q > 0 ? q - 1 : LS - 1;
          co = q > 0 ? R(-1) : m;
        } else {
          qn = q < LS - 1 ? q + 1 : 0;
          co = q < LS - 1 ? R(-1) : m;
        }
        res[q].re = fma(d, row[q].re, co * row[qn].re);
        res[q].im = fma(d, row[q].im, co * row[qn].im);
      }
#pragma unroll
      for (int q = 0; q < LS; q++) row[q] = res[q];
    }
#pragma unroll
    for (int q = 0; q < LS; q++) rp[q] = row[q];
  }
  __syncthreads();
  S* dst = out + base;
  for (int e = tid; e < nr * LS; e += 128) {
    const int r = e / LS, q = e - r * LS;
    st_c(dst + e, tile[r * (LS + 1) + q]);
  }
}

}  // namespace dwfk

#include "dhop_pair.cuh"

namespace dwfk {

template <int LS>
struct HopShape {
  static constexpr int SB = (LS >= 16) ? 8 : (128 / LS);
};

// Tuning variants of the hopping kernel: (register cap, prefetch).  Variant 0
// is the uncapped kernel; the autotuner (dwf_autotune) times the rest on the
// context's lattice and keeps the fastest per precision.
static_assert(DWF_HOP_VARIANTS == 26, "variant table below");
__host__ __device__ constexpr int hop_variant_regs(int v) {
  return v == 0 ? 0 : v == 1 ? 96 : v == 2 ? 80 : v == 3 ? 64 : v == 4 ? 128 : v == 5 ? 96 : v == 6 ? 64 : v == 7 ? 80
         : v == 8 ? 64 : v == 9 ? 80 : v == 10 ? 128 : v == 11 ? 112 : v == 12 ? 96 : v == 13 ? 0
         : v == 14 ? 64 : v == 15 ? 80 : v == 16 ? 64 : v == 17 ? 80 : v == 18 ? 56 : v == 19 ? 48
         : v == 23 ? 64 : v == 24 ? 64 : v == 25 ? 80 : 0;
}
// L2 prefetch distance of the scalar kernel in waves of resident CTAs
// (variants 23-25)
__host__ __device__ constexpr int hop_variant_l2pf(int v) { return v == 23 ? 1 : v == 24 ? 2 : v == 25 ? 1 : 0; }
// s-pair kernel with asynchronous shared-memory staging, neighbours in flight
// per thread (variants 20-22)
__host__ __device__ constexpr int hop_variant_depth(int v) { return v == 20 ? 8 : v == 21 ? 4 : v == 22 ? 2 : 0; }
// rows of sites per CTA (variants 14-17: scalar kernel on 2 or 4 y-rows)
__host__ __device__ constexpr int hop_variant_rows(int v) {
  return (v == 16 || v == 17) ? 4 : (v == 14 || v == 15) ? 2 : 1;
}
// 0: scalar, 1: scalar with neighbour prefetch, 2: packed FP32 (fma.rn.f32x2)
// on (re, im) pairs, 3: scalar on 2^4-hypercube tiles (8 output sites per
// CTA), 4: two s-slices per thread, packed FP32 over the s-pair
// (hop_kernel_pair)
__host__ __device__ constexpr int hop_variant_pf(int v) {
  return v >= 23 ? 0 : v >= 20 ? 4 : v >= 14 ? 0 : v >= 10 ? 4 : v >= 8 ? 3 : v >= 6 ? 2 : v >= 4 ? 1 : 0;
}  // 18, 19: scalar with 56 / 48 registers; 23-25: scalar with L2 prefetch

// Dynamic shared memory of one launch: links (SBC*72 complex, twice for the
// (re,re,-im,im) packed form), or the M_ee^-1 stage (SBC*12*(LS+1) complex)
// when the epilogue inverts; opted in above 48 KB once per instantiation.
template <auto Kern>
inline void hop_launch_smem(dim3 grid, int threads, size_t bytes, const HopParams& hp, cudaStream_t st) {
  static size_t opted = 48 * 1024;  // one per kernel instantiation
  if (bytes > opted) {
    cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    opted = bytes;
  }
  Kern<<<grid, threads, bytes, st>>>(hp);
}

template <int P, int LSV, int V>
inline void launch_hop_v(const HopParams& hp, dim3 grid, cudaStream_t st) {
  constexpr int SB = HopShape<LSV>::SB;
  constexpr int PF = hop_variant_pf(V);
  constexpr int RY = PF == 4 ? 1 : hop_variant_rows(V);
  constexpr size_t cb = sizeof(cpx<typename Prec<P>::R>);
  const size_t ub = (size_t)SB * RY * 72 * cb * (PF == 2 || PF == 4 ? 2 : 1);
  const size_t sb = hp.inv_mode ? (size_t)SB * RY * 12 * (LSV + 1) * cb : 0;
  const size_t bytes = ub > sb ? ub : sb;
  if constexpr (PF == 4 && hop_variant_depth(V) > 0) {
    constexpr int D = hop_variant_depth(V);
    hop_launch_smem<hop_kernel_pair<P, LSV, SB, hop_variant_regs(V), D>>(
        grid, LSV / 2 * SB, pair_smem_bytes<P, LSV, SB, D>(hp.inv_mode != 0), hp, st);
  } else if constexpr (PF == 4) {
    hop_launch_smem<hop_kernel_pair<P, LSV, SB, hop_variant_regs(V)>>(grid, LSV / 2 * SB, bytes, hp, st);
  } else if constexpr (hop_variant_l2pf(V) > 0) {
    // prefetch distance: the given number of waves of resident CTAs
    static int resident = 0;  // CTAs per GPU, one per instantiation
    if (!resident) {
      int dev = 0, nsm = 0, per = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, hop_kernel<P, LSV, SB, hop_variant_regs(V), PF, RY>,
                                                    LSV * SB * RY, bytes);
      resident = nsm * (per > 0 ? per : 1);
      if (resident < 1) resident = 1;
    }
    HopParams h2 = hp;
    h2.l2pf = hop_variant_l2pf(V) * resident;
    hop_launch_smem<hop_kernel<P, LSV, SB, hop_variant_regs(V), PF, RY>>(grid, LSV * SB * RY, bytes, h2, st);
  } else {
    hop_launch_smem<hop_kernel<P, LSV, SB, hop_variant_regs(V), PF, RY>>(grid, LSV * SB * RY, bytes, hp, st);
  }
}

template <int P, int LSV>
inline int launch_hop_ls(const HopParams& hp, dim3 grid, int variant, cudaStream_t st) {
  // FP64 is ALU-bound and the small-Ls cases are test sizes: one variant.
  if constexpr (P == DWF_F64 || LSV < 16) {
    launch_hop_v<P, LSV, 0>(hp, grid, st);
  } else if constexpr (P == DWF_P_DF) {
    // float-float: the plain kernel with register caps 96 / 80 / 64 (more
    // resident warps for its long dependent FP32 chains)
    switch (variant) {
      case 1: launch_hop_v<P, LSV, 1>(hp, grid, st); break;
      case 2: launch_hop_v<P, LSV, 2>(hp, grid, st); break;
      case 3: launch_hop_v<P, LSV, 3>(hp, grid, st); break;
      default: launch_hop_v<P, LSV, 0>(hp, grid, st); break;
    }
  } else {
    switch (variant) {
      case 1: launch_hop_v<P, LSV, 1>(hp, grid, st); break;
      case 2: launch_hop_v<P, LSV, 2>(hp, grid, st); break;
      case 3: launch_hop_v<P, LSV, 3>(hp, grid, st); break;
      case 4: launch_hop_v<P, LSV, 4>(hp, grid, st); break;
      case 5: launch_hop_v<P, LSV, 5>(hp, grid, st); break;
      case 6: launch_hop_v<P, LSV, 6>(hp, grid, st); break;
      case 7: launch_hop_v<P, LSV, 7>(hp, grid, st); break;
      case 8: launch_hop_v<P, LSV, 8>(hp, grid, st); break;
      case 9: launch_hop_v<P, LSV, 9>(hp, grid, st); break;
      case 10: launch_hop_v<P, LSV, 10>(hp, grid, st); break;
      case 11: launch_hop_v<P, LSV, 11>(hp, grid, st); break;
      case 12: launch_hop_v<P, LSV, 12>(hp, grid, st); break;
      case 13: launch_hop_v<P, LSV, 13>(hp, grid, st); break;
      case 14: launch_hop_v<P, LSV, 14>(hp, grid, st); break;
      case 15: launch_hop_v<P, LSV, 15>(hp, grid, st); break;
      case 16: launch_hop_v<P, LSV, 16>(hp, grid, st); break;
      case 17: launch_hop_v<P, LSV, 17>(hp, grid, st); break;
      case 18: launch_hop_v<P, LSV, 18>(hp, grid, st); break;
      case 19: launch_hop_v<P, LSV, 19>(hp, grid, st); break;
      case 20: launch_hop_v<P, LSV, 20>(hp, grid, st); break;
      case 21: launch_hop_v<P, LSV, 21>(hp, grid, st); break;
      case 22: launch_hop_v<P, LSV, 22>(hp, grid, st); break;
      case 23: launch_hop_v<P, LSV, 23>(hp, grid, st); break;
      case 24: launch_hop_v<P, LSV, 24>(hp, grid, st); break;
      case 25: launch_hop_v<P, LSV, 25>(hp, grid, st); break;
      default: launch_hop_v<P, LSV, 0>(hp, grid, st); break;
    }
  }
  return DWF_OK;
}

template <int P>
int launch_hop_prec(const HopParams& hp, int Ls, int nrhs, int variant, cudaStream_t st, int* nblocks) {
  dim3 grid;
  grid.y = nrhs;
  grid.z = 1;
#define DWF_HOP_CASE(LSV)                                                        \
  case LSV: {                                                                    \
    constexpr int SB = HopShape<LSV>::SB;                                        \
    const int ry = (P == DWF_F64 || P == DWF_P_DF || LSV < 16) ? 1 : hop_variant_rows(variant); \
    if (ry > 1 && (hp.Lxh % SB || hp.L1 % ry)) return DWF_EINVAL;                \
    grid.x = (hp.Vh + SB * ry - 1) / (SB * ry);                                  \
    if (nblocks) *nblocks = grid.x * grid.y;                                     \
    return launch_hop_ls<P, LSV>(hp, grid, variant, st);                         \
  }
  switch (Ls) {
    DWF_HOP_CASE(4)
    DWF_HOP_CASE(8)
    DWF_HOP_CASE(16)
    DWF_HOP_CASE(24)
    default:
      return DWF_EINVAL;
  }
#undef DWF_HOP_CASE
}

template <int P>
int launch_mooee_prec(void* out, const void* in, const HopParams& hp, int dagger, int inverse,
                      int Ls, int nrhs, long long rhs_stride, cudaStream_t st) {
  typedef typename Prec<P>::S S;
#define DWF_MOO_CASE(LSV)                                                                         \
  case LSV: {                                                                                     \
    constexpr int RB = MooRows<P, LSV>::v;                                                        \
    dim3 grid((unsigned)((hp.Vh * 12LL + RB - 1) / RB), nrhs, 1);                                 \
    mooee_kernel<P, LSV><<<grid, 128, 0, st>>>((S*)out, (const S*)in, hp.Vh, dagger, inverse,      \
                                               rhs_stride, hp);                                   \
    return DWF_OK;                                                                                \
  }
  switch (Ls) {
    DWF_MOO_CASE(4)
    DWF_MOO_CASE(8)
    DWF_MOO_CASE(16)
    DWF_MOO_CASE(24)
    default:
      return DWF_EINVAL;
  }
#undef DWF_MOO_CASE
}

}  // namespace dwfk

// Per-precision entry points (defined in dhop_f64.cu, dhop_f32.cu, dhop_f16.cu).
int dwf_launch_hop_f64(const dwfk::HopParams& hp, int Ls, int nrhs, int variant, cudaStream_t st, int* nb);
int dwf_launch_hop_f32(const dwfk::HopParams& hp, int Ls, int nrhs, int variant, cudaStream_t st, int* nb);
int dwf_launch_hop_f16(const dwfk::HopParams& hp, int Ls, int nrhs, int variant, cudaStream_t st, int* nb);
// FP64 storage, float-float arithmetic (dhop_df.cu)
int dwf_launch_hop_df(const dwfk::HopParams& hp, int Ls, int nrhs, int variant, cudaStream_t st, int* nb);
int dwf_launch_mooee_f64(void* out, const void* in, const dwfk::HopParams& hp, int dagger,
                         int inverse, int Ls, int nrhs, long long rs, cudaStream_t st);
int dwf_launch_mooee_f32(void* out, const void* in, const dwfk::HopParams& hp, int dagger,
                         int inverse, int Ls, int nrhs, long long rs, cudaStream_t st);
int dwf_launch_mooee_f16(void* out, const void* in, const dwfk::HopParams& hp, int dagger,
                         int inverse, int Ls, int nrhs, long long rs, cudaStream_t st);
