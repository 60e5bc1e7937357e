// Hopping term with two s-slices per thread and packed FP32 arithmetic over
// the pair (s, s+1) (fma.rn.f32x2 on sm_100+): D_hop is diagonal in s
// (Sec. 2, Eq. 2), so the same link multiplies both slices and every
// operation of the spin projection, the SU(3) multiply and the
// reconstruction is one packed instruction for two output sites.
//
// Registers hold (value at s, value at s+1) pairs, real and imaginary parts
// in separate pairs; a neighbour component is one 16-byte load (FP32; 8 bytes
// for FP16 storage) of the two consecutive complex numbers.  Links sit in
// shared memory as (re, re, im, im) so one 16-byte load yields both
// broadcast pairs.  The epilogues are those of hop_kernel (same HopParams).
#pragma once

#include <type_traits>

namespace dwfk {

template <int P>
struct PairIO;
template <>
struct PairIO<DWF_F32> {
  static __device__ __forceinline__ void ld(const float2* p, f2p& re, f2p& im) {
    const float4 v = *(const float4*)p;
    re = pk2(v.x, v.z);
    im = pk2(v.y, v.w);
  }
  static __device__ __forceinline__ void st(float2* p, f2p re, f2p im) {
    float a, b, c, d;
    upk2(re, a, c);
    upk2(im, b, d);
    *(float4*)p = make_float4(a, b, c, d);
  }
};
template <>
struct PairIO<DWF_F16S> {
  static __device__ __forceinline__ void ld(const __half2* p, f2p& re, f2p& im) {
    const uint2 v = *(const uint2*)p;
    __half2 h0, h1;
    memcpy(&h0, &v.x, 4);
    memcpy(&h1, &v.y, 4);
    const float2 f0 = __half22float2(h0), f1 = __half22float2(h1);
    re = pk2(f0.x, f1.x);
    im = pk2(f0.y, f1.y);
  }
  static __device__ __forceinline__ void st(__half2* p, f2p re, f2p im) {
    float a, b, c, d;
    upk2(re, a, c);
    upk2(im, b, d);
    const __half2 h0 = __floats2half2_rn(a, b), h1 = __floats2half2_rn(c, d);
    uint2 v;
    memcpy(&v.x, &h0, 4);
    memcpy(&v.y, &h1, 4);
    *(uint2*)p = v;
  }
};

__device__ __forceinline__ f2p mul2(f2p a, f2p b) {
  f2p d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// acc += (1 - sg gamma_mu) U psi on an s-pair; SG = (sg, sg), NSG = -SG,
// NEG = (-1, -1).  Same algebra as hop_dir (chiral basis).
template <int MU>
__device__ __forceinline__ void hop_dir_pair(f2p (&ar)[12], f2p (&ai)[12], const f2p (&pr)[12],
                                             const f2p (&pi)[12], const float4* __restrict__ U, f2p SG,
                                             f2p NSG, f2p NEG) {
  f2p h0r[3], h0i[3], h1r[3], h1i[3], n0i[3], n1i[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const int q0 = c, q1 = 3 + c, q2 = 6 + c, q3 = 9 + c;
    if (MU == 0) {  // h0 = p0 + s i p3, h1 = p1 + s i p2
      h0r[c] = fma2(NSG, pi[q3], pr[q0]);
      h0i[c] = fma2(SG, pr[q3], pi[q0]);
      h1r[c] = fma2(NSG, pi[q2], pr[q1]);
      h1i[c] = fma2(SG, pr[q2], pi[q1]);
    } else if (MU == 1) {  // h0 = p0 + s p3, h1 = p1 - s p2
      h0r[c] = fma2(SG, pr[q3], pr[q0]);
      h0i[c] = fma2(SG, pi[q3], pi[q0]);
      h1r[c] = fma2(NSG, pr[q2], pr[q1]);
      h1i[c] = fma2(NSG, pi[q2], pi[q1]);
    } else if (MU == 2) {  // h0 = p0 + s i p2, h1 = p1 - s i p3
      h0r[c] = fma2(NSG, pi[q2], pr[q0]);
      h0i[c] = fma2(SG, pr[q2], pi[q0]);
      h1r[c] = fma2(SG, pi[q3], pr[q1]);
      h1i[c] = fma2(NSG, pr[q3], pi[q1]);
    } else {  // h0 = p0 - s p2, h1 = p1 - s p3
      h0r[c] = fma2(NSG, pr[q2], pr[q0]);
      h0i[c] = fma2(NSG, pi[q2], pi[q0]);
      h1r[c] = fma2(NSG, pr[q3], pr[q1]);
      h1i[c] = fma2(NSG, pi[q3], pi[q1]);
    }
    n0i[c] = mul2(NEG, h0i[c]);
    n1i[c] = mul2(NEG, h1i[c]);
  }
#pragma unroll
  for (int a = 0; a < 3; a++) {
    f2p g0r = 0ull, g0i = 0ull, g1r = 0ull, g1i = 0ull;
#pragma unroll
    for (int b = 0; b < 3; b++) {
      const float4 u = U[a * 3 + b];
      const f2p ur = pk2(u.x, u.y), ui = pk2(u.z, u.w);
      g0r = fma2(ur, h0r[b], g0r);
      g0r = fma2(ui, n0i[b], g0r);
      g0i = fma2(ur, h0i[b], g0i);
      g0i = fma2(ui, h0r[b], g0i);
      g1r = fma2(ur, h1r[b], g1r);
      g1r = fma2(ui, n1i[b], g1r);
      g1i = fma2(ur, h1i[b], g1i);
      g1i = fma2(ui, h1r[b], g1i);
    }
    ar[a] = add2(ar[a], g0r);
    ai[a] = add2(ai[a], g0i);
    ar[3 + a] = add2(ar[3 + a], g1r);
    ai[3 + a] = add2(ai[3 + a], g1i);
    if (MU == 0) {  // lower: -s i g1, -s i g0
      ar[6 + a] = fma2(SG, g1i, ar[6 + a]);
      ai[6 + a] = fma2(NSG, g1r, ai[6 + a]);
      ar[9 + a] = fma2(SG, g0i, ar[9 + a]);
      ai[9 + a] = fma2(NSG, g0r, ai[9 + a]);
    } else if (MU == 1) {  // -s g1, s g0
      ar[6 + a] = fma2(NSG, g1r, ar[6 + a]);
      ai[6 + a] = fma2(NSG, g1i, ai[6 + a]);
      ar[9 + a] = fma2(SG, g0r, ar[9 + a]);
      ai[9 + a] = fma2(SG, g0i, ai[9 + a]);
    } else if (MU == 2) {  // -s i g0, s i g1
      ar[6 + a] = fma2(SG, g0i, ar[6 + a]);
      ai[6 + a] = fma2(NSG, g0r, ai[6 + a]);
      ar[9 + a] = fma2(NSG, g1i, ar[9 + a]);
      ai[9 + a] = fma2(SG, g1r, ai[9 + a]);
    } else {  // -s g0, -s g1
      ar[6 + a] = fma2(NSG, g0r, ar[6 + a]);
      ai[6 + a] = fma2(NSG, g0i, ai[6 + a]);
      ar[9 + a] = fma2(NSG, g1r, ar[9 + a]);
      ai[9 + a] = fma2(NSG, g1i, ai[9 + a]);
    }
  }
}

template <int P, int LS>
__device__ __forceinline__ void load_pair(f2p (&pr)[12], f2p (&pi)[12], const typename Prec<P>::S* __restrict__ base) {
#pragma unroll
  for (int c = 0; c < 12; c++) PairIO<P>::ld(base + c * LS, pr[c], pi[c]);
}

// Asynchronous staging (D > 0): each thread copies its own s-pair of every
// neighbour component straight from global to shared memory (cp.async, no
// register staging), up to D neighbours in flight per thread, and reads each
// back when its copy group has landed.  Shared memory, not the register file,
// then bounds the bytes in flight.  Slot layout [slot][component][thread] so
// that a warp's reads are contiguous.
template <int P>
struct PairBytes {
  static constexpr int v = P == DWF_F32 ? 16 : 8;
};
template <int B>
__device__ __forceinline__ void cp_async_bytes(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (B == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
  }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
template <int P>
__device__ __forceinline__ void read_staged(const unsigned char* slot, int nt, int tid, f2p (&pr)[12], f2p (&pi)[12]) {
#pragma unroll
  for (int c = 0; c < 12; c++) {
    const typename Prec<P>::S* e =
        (const typename Prec<P>::S*)(slot + ((size_t)c * nt + tid) * PairBytes<P>::v);
    PairIO<P>::ld(e, pr[c], pi[c]);
  }
}

// Shared memory of one launch of hop_kernel_pair<.., D> (bytes).
template <int P, int LS, int SB, int D>
__host__ __device__ constexpr size_t pair_smem_bytes(bool inv) {
  return (size_t)SB * 72 * 16 +
         (D > 0 ? ((size_t)D * 12 * (LS / 2 * SB) * PairBytes<P>::v > (inv ? (size_t)SB * 12 * (LS + 1) * 8 : 0)
                       ? (size_t)D * 12 * (LS / 2 * SB) * PairBytes<P>::v
                       : (inv ? (size_t)SB * 12 * (LS + 1) * 8 : 0))
                 : 0);
}

// One CTA: SB consecutive checkerboard sites x LS/2 threads (s-pairs).
// D = 0: neighbours loaded into registers one at a time; D > 0: staged
// asynchronously in shared memory, D neighbours deep.
template <int P, int LS, int SB, int REGS, int D = 0>
__global__ void __launch_bounds__(LS / 2 * SB, (HopMinBlocks<LS / 2, SB, REGS>::v)) hop_kernel_pair(const HopParams p) {
  static_assert(P != DWF_F64, "packed FP32 kernel");
  static_assert(LS % 2 == 0, "Ls must be even");
  typedef typename Prec<P>::S S;
  typedef typename Prec<P>::LS LT;
  constexpr int TPS = LS / 2;
  constexpr int NT = TPS * SB;
  // dynamic shared memory: links during the hop, then (inv_mode) the
  // M_ee^-1 stage in the same bytes; with D > 0 the staging slots follow the
  // links and the M_ee^-1 stage reuses the slots (sized by the launcher)
  float4* sU = (float4*)hop_dyn_smem;
  unsigned char* stg = hop_dyn_smem + (D > 0 ? SB * 72 * 16 : 0);
  cpx<float>* stage = (cpx<float>*)stg;
  constexpr int SLOT = 12 * NT * PairBytes<P>::v;
  __shared__ double red[NT / 32 + 1];

  const int tid = threadIdx.x;
  const int sl = tid / TPS;
  const int q = tid - sl * TPS;
  const int s0 = 2 * q;
  const int zc = p.zc;
  int site0;
  if (zc < p.L2 && (p.Lxh % SB) == 0) {
    const int nseg = p.Lxh / SB;
    int r = blockIdx.x;
    const int seg = r % nseg;
    r /= nseg;
    const int yy = r % p.L1;
    r /= p.L1;
    const int zl = r % zc;
    r /= zc;
    const int tt = r % p.L3;
    const int zz = (r / p.L3) * zc + zl;
    site0 = ((tt * p.L2 + zz) * p.L1 + yy) * p.Lxh + seg * SB;
  } else {
    site0 = blockIdx.x * SB;
  }
  const int rhs = blockIdx.y;
  const int site = site0 + sl;
  const bool active = site < p.Vh;

  // coordinates and the first neighbour are fetched before the link barrier
  int rem = (active ? site : 0) / p.Lxh;
  const int xh = (active ? site : 0) - rem * p.Lxh;
  const int y = rem % p.L1;
  rem /= p.L1;
  const int z = rem % p.L2;
  const int t = rem / p.L2;
  const int x = 2 * xh + ((y + z + t + p.out_parity) & 1);
  const S* in = (const S*)p.in + (size_t)rhs * p.rhs_stride + s0;
  const int Lxh = p.Lxh, L1 = p.L1, L2 = p.L2;
  auto cbi = [&](int X, int Y, int Z, int T) { return ((T * L2 + Z) * L1 + Y) * Lxh + (X >> 1); };
  const int xp = (x + 1 == p.L0) ? 0 : x + 1, xm = (x == 0) ? p.L0 - 1 : x - 1;
  const int yp = (y + 1 == p.L1) ? 0 : y + 1, ym = (y == 0) ? p.L1 - 1 : y - 1;
  const int zp = (z + 1 == p.L2) ? 0 : z + 1, zm = (z == 0) ? p.L2 - 1 : z - 1;
  const int tp = (t + 1 == p.L3) ? 0 : t + 1, tm = (t == 0) ? p.L3 - 1 : t - 1;
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
  f2p pr[12], pi[12];
  auto issue = [&](int d) {  // D > 0: one copy group per neighbour
    unsigned char* slot = stg + (d % (D > 0 ? D : 1)) * SLOT;
    const S* src = nbp(d);
#pragma unroll
    for (int c = 0; c < 12; c++)
      cp_async_bytes<PairBytes<P>::v>(slot + ((size_t)c * NT + tid) * PairBytes<P>::v, src + c * LS);
    cp_async_commit();
  };
  if (active) {
    if constexpr (D > 0) {
#pragma unroll
      for (int d = 0; d < (D < 8 ? D : 8); d++) issue(d);
    } else {
      load_pair<P, LS>(pr, pi, nbp(0));
    }
  }
  {
    const LT* gl = (const LT*)p.links + (size_t)site0 * 72;
    const int n = min(SB, p.Vh - site0) * 72;
    for (int i = tid; i < n; i += NT) {
      const LT v = gl[i];
      sU[i] = make_float4((float)v.x, (float)v.x, (float)v.y, (float)v.y);
    }
  }
  __syncthreads();

  f2p vr[12], vi[12];
#pragma unroll
  for (int c = 0; c < 12; c++) vr[c] = vi[c] = 0ull;

  if (active) {
    const float4* U = sU + sl * 72;
    const float sgf = p.sg;
    const f2p SG = pk2(sgf, sgf), NSG = pk2(-sgf, -sgf), NEG = pk2(-1.f, -1.f);
    if constexpr (D > 0) {
      // neighbour d is in slot d % D; before reading it, at most
      // min(7, d + D - 1) - d later groups may still be in flight
      auto step = [&](auto dc) {
        constexpr int d = decltype(dc)::value;
        constexpr int later = (d + D - 1 < 7 ? d + D - 1 : 7) - d;
        cp_async_wait<later>();
        read_staged<P>(stg + (d % D) * SLOT, NT, tid, pr, pi);
        if (d & 1)
          hop_dir_pair<d / 2>(vr, vi, pr, pi, U + d * 9, NSG, SG, NEG);
        else
          hop_dir_pair<d / 2>(vr, vi, pr, pi, U + d * 9, SG, NSG, NEG);
        if (d + D < 8) issue(d + D);  // the slot's values are consumed
      };
      step(std::integral_constant<int, 0>());
      step(std::integral_constant<int, 1>());
      step(std::integral_constant<int, 2>());
      step(std::integral_constant<int, 3>());
      step(std::integral_constant<int, 4>());
      step(std::integral_constant<int, 5>());
      step(std::integral_constant<int, 6>());
      step(std::integral_constant<int, 7>());
    } else {
      hop_dir_pair<0>(vr, vi, pr, pi, U + 0 * 9, SG, NSG, NEG);  // neighbour 0 loaded above
      load_pair<P, LS>(pr, pi, nbp(1));
      hop_dir_pair<0>(vr, vi, pr, pi, U + 1 * 9, NSG, SG, NEG);
      load_pair<P, LS>(pr, pi, nbp(2));
      hop_dir_pair<1>(vr, vi, pr, pi, U + 2 * 9, SG, NSG, NEG);
      load_pair<P, LS>(pr, pi, nbp(3));
      hop_dir_pair<1>(vr, vi, pr, pi, U + 3 * 9, NSG, SG, NEG);
      load_pair<P, LS>(pr, pi, nbp(4));
      hop_dir_pair<2>(vr, vi, pr, pi, U + 4 * 9, SG, NSG, NEG);
      load_pair<P, LS>(pr, pi, nbp(5));
      hop_dir_pair<2>(vr, vi, pr, pi, U + 5 * 9, NSG, SG, NEG);
      load_pair<P, LS>(pr, pi, nbp(6));
      hop_dir_pair<3>(vr, vi, pr, pi, U + 6 * 9, SG, NSG, NEG);
      load_pair<P, LS>(pr, pi, nbp(7));
      hop_dir_pair<3>(vr, vi, pr, pi, U + 7 * 9, NSG, SG, NEG);
    }

    const float al = (float)p.alpha;
    const f2p AL = pk2(al, al);
#pragma unroll
    for (int c = 0; c < 12; c++) {
      vr[c] = mul2(AL, vr[c]);
      vi[c] = mul2(AL, vi[c]);
    }
    if (p.aux_mode) {
      const S* aux = (const S*)p.aux + (size_t)rhs * p.rhs_stride + (size_t)site * 12 * LS;
      if (p.aux_mode == 1) {
#pragma unroll
        for (int c = 0; c < 12; c++) {
          f2p ar, ai;
          PairIO<P>::ld(aux + c * LS + s0, ar, ai);
          vr[c] = add2(vr[c], ar);
          vi[c] = add2(vi[c], ai);
        }
      } else {
        // M psi_s = d psi_s + co psi_{s-+1}: chirality + (spins 0,1) of M
        // couples s-1 (coefficient m at the wall s = 0), chirality - couples
        // s+1 (m at s = Ls-1); M^dag swaps the two rules.
        const bool dagM = p.aux_mode == 3;
        const float d = (float)p.d, m = (float)p.m[rhs];
        const f2p D = pk2(d, d);
        const int sm0 = q > 0 ? s0 - 1 : LS - 1;  // s-1 of the first slice
        const int sp1 = s0 + 2 < LS ? s0 + 2 : 0;  // s+1 of the second slice
        const f2p COL = pk2(q > 0 ? -1.f : m, -1.f);
        const f2p COU = pk2(-1.f, s0 + 2 < LS ? -1.f : m);
#pragma unroll
        for (int c = 0; c < 12; c++) {
          const bool lower = (c < 6) != dagM;
          f2p ar, ai;
          PairIO<P>::ld(aux + c * LS + s0, ar, ai);
          const cpx<float> e = ld_c(aux + c * LS + (lower ? sm0 : sp1));
          float a0r, a1r, a0i, a1i;
          upk2(ar, a0r, a1r);
          upk2(ai, a0i, a1i);
          const f2p nr = lower ? pk2(e.re, a0r) : pk2(a1r, e.re);
          const f2p ni = lower ? pk2(e.im, a0i) : pk2(a1i, e.im);
          const f2p CO = lower ? COL : COU;
          vr[c] = add2(vr[c], fma2(D, ar, mul2(CO, nr)));
          vi[c] = add2(vi[c], fma2(D, ai, mul2(CO, ni)));
        }
      }
    }
  }

  if (p.inv_mode) {
    __syncthreads();  // every thread is done with the links
    if (active) {
#pragma unroll
      for (int c = 0; c < 12; c++) {
        float a, b, e, f;
        upk2(vr[c], a, b);
        upk2(vi[c], e, f);
        stage[(sl * 12 + c) * (LS + 1) + s0] = cmake<float>(a, e);
        stage[(sl * 12 + c) * (LS + 1) + s0 + 1] = cmake<float>(b, f);
      }
    }
    __syncthreads();
    for (int w = tid; w < SB * 12; w += NT) {
      const int sl2 = w / 12, c2 = w - sl2 * 12;
      if (site0 + sl2 < p.Vh) {
        const bool fwd = (c2 < 6) != (p.inv_mode == 2);
        minv_row_inplace<float, LS>(stage + (sl2 * 12 + c2) * (LS + 1), fwd, (float)p.d, (float)p.m[rhs],
                                    (float)p.kappa[rhs], (float)p.dls1[rhs]);
      }
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int c = 0; c < 12; c++) {
        const cpx<float> a = stage[(sl * 12 + c) * (LS + 1) + s0];
        const cpx<float> b = stage[(sl * 12 + c) * (LS + 1) + s0 + 1];
        vr[c] = pk2(a.re, b.re);
        vi[c] = pk2(a.im, b.im);
      }
    }
  }

  if (p.cg_mode) {
    if (active) {
      const size_t off = (size_t)rhs * p.rhs_stride + (size_t)site * 12 * LS + s0;
      S* xs = (S*)p.cg_x + off;
      S* rs = (S*)p.cg_r + off;
      const S* ps = (const S*)p.cg_p + off;
      const float al = (float)p.cg_alpha[(size_t)rhs * p.cg_astride];
      const f2p AL = pk2(al, al), NAL = pk2(-al, -al);
      float2* xs32 = (float2*)p.cg_x + off;
      const bool x32 = (P == DWF_F16S) && p.cg_x32;
#pragma unroll
      for (int c = 0; c < 12; c++) {
        f2p xr, xi, rr, ri, pr, pi;
        if (x32)
          PairIO<DWF_F32>::ld(xs32 + c * LS, xr, xi);
        else
          PairIO<P>::ld(xs + c * LS, xr, xi);
        PairIO<P>::ld(rs + c * LS, rr, ri);
        PairIO<P>::ld(ps + c * LS, pr, pi);
        xr = fma2(AL, pr, xr);
        xi = fma2(AL, pi, xi);
        rr = fma2(NAL, vr[c], rr);
        ri = fma2(NAL, vi[c], ri);
        if (x32)
          PairIO<DWF_F32>::st(xs32 + c * LS, xr, xi);
        else
          PairIO<P>::st(xs + c * LS, xr, xi);
        PairIO<P>::st(rs + c * LS, rr, ri);
        vr[c] = rr;
        vi[c] = ri;
      }
    }
  } else if (active && p.cheb_mode) {
    // tp = ta v + tb x - tp; acc += cacc tp, on the pair's store positions
    const size_t base = (size_t)rhs * p.rhs_stride + (size_t)site * 12 * LS;
    const int so = p.g5r5 ? LS - 2 - s0 : s0;
    const S* cx = (const S*)p.cheb_x + base;
    S* ct = (S*)p.cheb_tp + base;
    S* ca = p.cheb_acc ? (S*)p.cheb_acc + base : nullptr;
    const float ta = (float)p.cheb_ta, tb = (float)p.cheb_tb, cc = (float)p.cheb_cacc;
    const f2p TA = pk2(ta, ta), TB = pk2(tb, tb), CC = pk2(cc, cc), NEG = pk2(-1.f, -1.f);
#pragma unroll
    for (int c = 0; c < 12; c++) {
      f2p r = vr[c], i = vi[c];
      if (p.g5r5) {
        r = swp2(r);
        i = swp2(i);
        if (c >= 6) {
          r = mul2(NEG, r);
          i = mul2(NEG, i);
        }
      }
      f2p xr, xi, tr, ti;
      PairIO<P>::ld(cx + c * LS + so, xr, xi);
      PairIO<P>::ld(ct + c * LS + so, tr, ti);
      const f2p wr = fma2(TA, r, fma2(TB, xr, mul2(NEG, tr)));
      const f2p wi = fma2(TA, i, fma2(TB, xi, mul2(NEG, ti)));
      PairIO<P>::st(ct + c * LS + so, wr, wi);
      if (ca) {
        f2p ar, ai;
        PairIO<P>::ld(ca + c * LS + so, ar, ai);
        PairIO<P>::st(ca + c * LS + so, fma2(CC, wr, ar), fma2(CC, wi, ai));
      }
    }
  } else if (active) {
    S* out = (S*)p.out + (size_t)rhs * p.rhs_stride + (size_t)site * 12 * LS;
    if (p.g5r5) {
      // slice s goes to Ls-1-s: the pair (s0, s0+1) lands on (Ls-2-s0, Ls-1-s0) swapped
      const int so = LS - 2 - s0;
      const f2p NEG = pk2(-1.f, -1.f);
#pragma unroll
      for (int c = 0; c < 12; c++) {
        f2p r = swp2(vr[c]), i = swp2(vi[c]);
        if (c >= 6) {
          r = mul2(NEG, r);
          i = mul2(NEG, i);
        }
        PairIO<P>::st(out + c * LS + so, r, i);
      }
    } else {
#pragma unroll
      for (int c = 0; c < 12; c++) PairIO<P>::st(out + c * LS + s0, vr[c], vi[c]);
    }
  }

  if (p.reduce) {
    PartialSum<float> ps;
    if (active) {
#pragma unroll
      for (int c = 0; c < 12; c++) {
        float a, b, e, f;
        upk2(vr[c], a, b);
        upk2(vi[c], e, f);
        ps.add(fmaf(a, a, b * b));
        ps.add(fmaf(e, e, f * f));
      }
    }
    double acc = ps.value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();
    if (tid == 0) {
      double tot = 0.0;
      for (int i = 0; i < (NT + 31) / 32; i++) tot += red[i];
      p.partials[blockIdx.y * gridDim.x + blockIdx.x] = tot;
    }
  }
}

}  // namespace dwfk
