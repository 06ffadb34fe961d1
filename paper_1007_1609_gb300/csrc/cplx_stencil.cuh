// cplx_stencil.cuh -- one application of the general lattice Hamiltonian of
// Eq. 2 (complex hoppings with Peierls phases, optional next-nearest
// neighbours, on-site or nearest-neighbour bond pairing) to a site of a
// lattice row of a column slab held in shared memory:
//   u' = e u + D v - sum_d t_d u_d + sum_{d<4} B_d v_d - u_old       (electron row)
//   v' = conj(D) u - e v + sum_d conj(t_d) v_d + sum_{d<4} conj(B_d) u_d - v_old
// with e = 2(eps - mu)/a, D = 2 Delta/a, t_d = 2 t_{s,d}/a, B_d = 2 Delta_{s,d}/a.
// A site stores only its forward hoppings (+x, +y, +x+y, -x+y) and bonds
// (+x, +y); the backward ones are those of the left, lower and diagonal
// neighbours, conjugated for the hoppings.  Shared by the one-step kernel
// (step_cplx.cu) and the two-step pass (step_cplx_multi.cu).
//
// FP32: a complex64 element (re, im) is one packed pair of the f32x2
// instructions (f32x2.cuh), two FP32 operations each.  A product c z with a
// complex coefficient c splits into
// A += (c.re, c.re) z and S += (c.im, c.im) z, combined once per element at
// the end: c z = (A.x - S.y, A.y + S.x) and conj(c) z = (A.x + S.y, A.y - S.x).
// Half the FMA instructions of four scalar FMAs per complex multiply-add, and
// the dependent chains are half as long (A and S accumulate independently).
#pragma once

#include <type_traits>

#include "f32x2.cuh"
#include "internal.h"

namespace cbdg {
namespace cx {

template <typename S>
struct Cx {
  S re, im;
};
template <typename S>
__device__ __forceinline__ Cx<S> cmul(Cx<S> a, Cx<S> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename S>
__device__ __forceinline__ Cx<S> cmulc(Cx<S> a, Cx<S> b) {  // conj(a) * b
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <typename S>
__device__ __forceinline__ Cx<S> cadd(Cx<S> a, Cx<S> b) {
  return {a.re + b.re, a.im + b.im};
}
template <typename S>
__device__ __forceinline__ Cx<S> csub(Cx<S> a, Cx<S> b) {
  return {a.re - b.re, a.im - b.im};
}

__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
// acc + a * b and acc + conj(a) * b, four FMAs each
template <typename S>
__device__ __forceinline__ Cx<S> cmac(Cx<S> acc, Cx<S> a, Cx<S> b) {
  return {fma_rn(a.re, b.re, fma_rn(-a.im, b.im, acc.re)), fma_rn(a.re, b.im, fma_rn(a.im, b.re, acc.im))};
}
template <typename S>
__device__ __forceinline__ Cx<S> cmacc(Cx<S> acc, Cx<S> a, Cx<S> b) {
  return {fma_rn(a.re, b.re, fma_rn(a.im, b.im, acc.re)), fma_rn(a.re, b.im, fma_rn(-a.im, b.re, acc.im))};
}
template <typename S>
__device__ __forceinline__ Cx<S> cneg(Cx<S> a) {
  return {-a.re, -a.im};
}

template <typename V, typename S>
__device__ __forceinline__ Cx<S> cget(const V &v, int j) {
  const S *p = reinterpret_cast<const S *>(&v);
  return {p[2 * j], p[2 * j + 1]};
}
template <typename V, typename S>
__device__ __forceinline__ void cset(V &v, int j, Cx<S> z) {
  S *p = reinterpret_cast<S *>(&v);
  p[2 * j] = z.re;
  p[2 * j + 1] = z.im;
}

template <typename S>
struct Pair;
template <>
struct Pair<float> {
  using T = float2;
};
template <>
struct Pair<double> {
  using T = double2;
};
// Complex field k of a site's parameters, one 8- or 16-byte load; p points at
// field 0 of the site inside its lattice row, fields are 2 Lx scalars apart
// (see internal.h).
template <typename S, bool LDG>
__device__ __forceinline__ Cx<S> pcx(const S *p, int k, int Lx) {
  using P = typename Pair<S>::T;
  const P *q = reinterpret_cast<const P *>(p + static_cast<size_t>(k) * 2 * Lx);
  const P v = LDG ? __ldg(q) : *q;
  return {v.x, v.y};
}


// The update of site x (neighbours xl, xr) for the VC complex columns of
// this thread: rows rm, rc, rp (y - 1, y, y + 1) of j_n and ro (row y of
// j_{n-1}) in the slab-row layout (electron sites, then hole sites at hb
// scalars, W complex columns per site, this thread's at `off`), parameter
// rows py0 (y) and py1 (y - 1).  Returns j_n's components u, v at x and the
// new un, vn.  LDG: parameters through the read-only cache (global memory).
template <typename S, typename V, int VC, int W, bool NNN, bool BOND, bool LDG>
__device__ __forceinline__ void site_step_scalar(const S *rm, const S *rc, const S *rp, const S *ro, const S *py0,
                                                 const S *py1, int x, int xl, int xr, int off, int hb, int Lx, V &u,
                                                 V &v, V &un, V &vn) {
    auto ld = [&](const S *row, int xx, int part) {
      return *reinterpret_cast<const V *>(row + part * hb + xx * W * 2 + off);
    };
    const S *pp = py0 + 2 * x;
    const S e = pcx<S, LDG>(pp, kCpE, Lx).re;
    const Cx<S> dl = pcx<S, LDG>(pp, kCpDelta, Lx);
    auto conj_ = [](Cx<S> z) { return Cx<S>{z.re, -z.im}; };
    // hopping of direction dd: forward from this site, backward from the neighbour
    auto hop_of = [&](int dd) -> Cx<S> {
      switch (dd) {
        case 0: return pcx<S, LDG>(pp, kCpHop + 0, Lx);
        case 1: return conj_(pcx<S, LDG>(py0 + 2 * xl, kCpHop + 0, Lx));
        case 2: return pcx<S, LDG>(pp, kCpHop + 1, Lx);
        case 3: return conj_(pcx<S, LDG>(py1 + 2 * x, kCpHop + 1, Lx));
        case 4: return pcx<S, LDG>(pp, kCpHop + 2, Lx);
        case 5: return conj_(pcx<S, LDG>(py1 + 2 * xl, kCpHop + 2, Lx));
        case 6: return conj_(pcx<S, LDG>(py1 + 2 * xr, kCpHop + 3, Lx));
        default: return pcx<S, LDG>(pp, kCpHop + 3, Lx);
      }
    };
    auto bond_of = [&](int dd) -> Cx<S> {
      switch (dd) {
        case 0: return pcx<S, LDG>(pp, kCpBond + 0, Lx);
        case 1: return pcx<S, LDG>(py0 + 2 * xl, kCpBond + 0, Lx);
        case 2: return pcx<S, LDG>(pp, kCpBond + 1, Lx);
        default: return pcx<S, LDG>(py1 + 2 * x, kCpBond + 1, Lx);
      }
    };
    // neighbour rows/columns per direction 0:+x 1:-x 2:+y 3:-y 4:+x+y 5:-x-y 6:+x-y 7:-x+y
    const S *nrow[8] = {rc, rc, rp, rm, rp, rm, rm, rp};
    const int ncol[8] = {xr, xl, x, x, xr, xl, xr, xl};
    u = ld(rc, x, 0);
    v = ld(rc, x, 1);
    const V uo = ld(ro, x, 0), vo = ld(ro, x, 1);
    // start from -j_{n-1} and the on-site terms:
    //   u' = e u + D v - u_old,  v' = conj(D) u - e v - v_old
#pragma unroll
    for (int j = 0; j < VC; ++j) {
      const Cx<S> uj = cget<V, S>(u, j), vj = cget<V, S>(v, j);
      const Cx<S> uoj = cget<V, S>(uo, j), voj = cget<V, S>(vo, j);
      const Cx<S> hu = cmac(Cx<S>{fma_rn(e, uj.re, -uoj.re), fma_rn(e, uj.im, -uoj.im)}, dl, vj);
      const Cx<S> hv = cmacc(Cx<S>{fma_rn(-e, vj.re, -voj.re), fma_rn(-e, vj.im, -voj.im)}, dl, uj);
      cset<V, S>(un, j, hu);
      cset<V, S>(vn, j, hv);
    }
#pragma unroll
    for (int dd = 0; dd < (NNN ? 8 : 4); ++dd) {
      const V ud = ld(nrow[dd], ncol[dd], 0), vd = ld(nrow[dd], ncol[dd], 1);
      const Cx<S> td = hop_of(dd), ntd = cneg(td);
      const Cx<S> bd = (BOND && dd < 4) ? bond_of(dd) : Cx<S>{0, 0};
#pragma unroll
      for (int j = 0; j < VC; ++j) {
        Cx<S> hu = cget<V, S>(un, j), hv = cget<V, S>(vn, j);
        // u' -= t_d u_d, v' += conj(t_d) v_d; bond pairing: u' += B_d v_d, v' += conj(B_d) u_d
        hu = cmac(hu, ntd, cget<V, S>(ud, j));
        hv = cmacc(hv, td, cget<V, S>(vd, j));
        if (BOND && dd < 4) {
          hu = cmac(hu, bd, cget<V, S>(vd, j));
          hv = cmacc(hv, bd, cget<V, S>(ud, j));
        }
        cset<V, S>(un, j, hu);
        cset<V, S>(vn, j, hv);
      }
    }
}

// The FP32 update of site_step_scalar with packed pairs (two complex64
// columns per float4).  Per element j of this thread:
//   u' = P_u - N_u with P_u = e u + D v + sum_{d<4} B_d v_d and
//        N_u = u_old + sum_d t_d u_d (both by the c z rule);
//   v' = P_v - e v - v_old with P_v = conj(D) u + sum_d conj(t_d) v_d
//        + sum_{d<4} conj(B_d) u_d (the conj(c) z rule).
template <int W, bool NNN, bool BOND, bool LDG>
__device__ __forceinline__ void site_step_f32x2(const float *rm, const float *rc, const float *rp, const float *ro,
                                                const float *py0, const float *py1, int x, int xl, int xr, int off,
                                                int hb, int Lx, float4 &u, float4 &v, float4 &un, float4 &vn) {
  auto ld = [&](const float *row, int xx, int part) {
    return *reinterpret_cast<const float4 *>(row + part * hb + xx * W * 2 + off);
  };
  auto lo = [](const float4 &q) { return f2lo(q); };
  auto hi = [](const float4 &q) { return f2hi(q); };
  const float *pp = py0 + 2 * x;
  const float e = pcx<float, LDG>(pp, kCpE, Lx).re;
  const Cx<float> dl = pcx<float, LDG>(pp, kCpDelta, Lx);
  auto conj_ = [](Cx<float> z) { return Cx<float>{z.re, -z.im}; };
  auto hop_of = [&](int dd) -> Cx<float> {
    switch (dd) {
      case 0: return pcx<float, LDG>(pp, kCpHop + 0, Lx);
      case 1: return conj_(pcx<float, LDG>(py0 + 2 * xl, kCpHop + 0, Lx));
      case 2: return pcx<float, LDG>(pp, kCpHop + 1, Lx);
      case 3: return conj_(pcx<float, LDG>(py1 + 2 * x, kCpHop + 1, Lx));
      case 4: return pcx<float, LDG>(pp, kCpHop + 2, Lx);
      case 5: return conj_(pcx<float, LDG>(py1 + 2 * xl, kCpHop + 2, Lx));
      case 6: return conj_(pcx<float, LDG>(py1 + 2 * xr, kCpHop + 3, Lx));
      default: return pcx<float, LDG>(pp, kCpHop + 3, Lx);
    }
  };
  auto bond_of = [&](int dd) -> Cx<float> {
    switch (dd) {
      case 0: return pcx<float, LDG>(pp, kCpBond + 0, Lx);
      case 1: return pcx<float, LDG>(py0 + 2 * xl, kCpBond + 0, Lx);
      case 2: return pcx<float, LDG>(pp, kCpBond + 1, Lx);
      default: return pcx<float, LDG>(py1 + 2 * x, kCpBond + 1, Lx);
    }
  };
  const float *nrow[8] = {rc, rc, rp, rm, rp, rm, rm, rp};
  const int ncol[8] = {xr, xl, x, x, xr, xl, xr, xl};
  u = ld(rc, x, 0);
  v = ld(rc, x, 1);
  const float4 uo = ld(ro, x, 0), vo = ld(ro, x, 1);
  const F2 z = f2pack(0.f, 0.f);
  const F2 be = f2bcast(e), bdr = f2bcast(dl.re), bdi = f2bcast(dl.im);
  const F2 uu[2] = {lo(u), hi(u)}, vv[2] = {lo(v), hi(v)};
  const F2 uop[2] = {lo(uo), hi(uo)}, vop[2] = {lo(vo), hi(vo)};
  F2 puA[2], puS[2], nuA[2], nuS[2], pvA[2], pvS[2], nv[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    puA[j] = f2fma(bdr, vv[j], f2fma(be, uu[j], z));
    puS[j] = f2fma(bdi, vv[j], z);
    pvA[j] = f2fma(bdr, uu[j], z);
    pvS[j] = f2fma(bdi, uu[j], z);
    nv[j] = f2fma(be, vv[j], vop[j]);
    nuA[j] = uop[j];
    nuS[j] = z;
  }
#pragma unroll
  for (int dd = 0; dd < (NNN ? 8 : 4); ++dd) {
    const float4 ud = ld(nrow[dd], ncol[dd], 0), vd = ld(nrow[dd], ncol[dd], 1);
    const F2 udp[2] = {lo(ud), hi(ud)}, vdp[2] = {lo(vd), hi(vd)};
    const Cx<float> td = hop_of(dd);
    const F2 btr = f2bcast(td.re), bti = f2bcast(td.im);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      nuA[j] = f2fma(btr, udp[j], nuA[j]);
      nuS[j] = f2fma(bti, udp[j], nuS[j]);
      pvA[j] = f2fma(btr, vdp[j], pvA[j]);
      pvS[j] = f2fma(bti, vdp[j], pvS[j]);
    }
    if (BOND && dd < 4) {
      const Cx<float> bd = bond_of(dd);
      const F2 bbr = f2bcast(bd.re), bbi = f2bcast(bd.im);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        puA[j] = f2fma(bbr, vdp[j], puA[j]);
        puS[j] = f2fma(bbi, vdp[j], puS[j]);
        pvA[j] = f2fma(bbr, udp[j], pvA[j]);
        pvS[j] = f2fma(bbi, udp[j], pvS[j]);
      }
    }
  }
  float o[2][4];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    float ax, ay, sx, sy;
    f2unpack(f2sub(puA[j], nuA[j]), ax, ay);
    f2unpack(f2sub(puS[j], nuS[j]), sx, sy);
    o[0][2 * j] = ax - sy;
    o[0][2 * j + 1] = ay + sx;
    f2unpack(f2sub(pvA[j], nv[j]), ax, ay);
    f2unpack(pvS[j], sx, sy);
    o[1][2 * j] = ax + sy;
    o[1][2 * j + 1] = ay - sx;
  }
  un = make_float4(o[0][0], o[0][1], o[0][2], o[0][3]);
  vn = make_float4(o[1][0], o[1][1], o[1][2], o[1][3]);
}

// The update of site x for this thread's VC complex columns (see
// site_step_scalar); FP32 takes the packed-pair form.
template <typename S, typename V, int VC, int W, bool NNN, bool BOND, bool LDG>
__device__ __forceinline__ void site_step(const S *rm, const S *rc, const S *rp, const S *ro, const S *py0,
                                          const S *py1, int x, int xl, int xr, int off, int hb, int Lx, V &u,
                                          V &v, V &un, V &vn) {
  if constexpr (std::is_same<S, float>::value && std::is_same<V, float4>::value && VC == 2)
    site_step_f32x2<W, NNN, BOND, LDG>(rm, rc, rp, ro, py0, py1, x, xl, xr, off, hb, Lx, u, v, un, vn);
  else
    site_step_scalar<S, V, VC, W, NNN, BOND, LDG>(rm, rc, rp, ro, py0, py1, x, xl, xr, off, hb, Lx, u, v, un, vn);
}

}  // namespace cx
}  // namespace cbdg
