// 2.5-D z-marching stencil kernels with shared-memory plane exchange.
//
// A block owns a 32 x 8 tile of (i, j) columns and walks planes k0..k1-1.
// The stencil input u (the iterate, or a value formed from several arrays,
// e.g. x + P e or D^-1 b / theta) is formed ONCE per point per plane by the
// thread that owns the point (halo points by designated threads) and written
// to one of three shared planes with a one-point halo; the in-plane
// neighbours come from shared memory, the z neighbours from a register queue.
// The raw loads of plane k+1 and the centre-only fields of plane k are issued
// one step ahead, so they are in flight while plane k is computed.  One
// __syncthreads per plane (three planes rotate, so a plane is never
// overwritten while a slow warp may still read it).
//
// Policy interface (Pol):
//   using R;                        compute type
//   struct Raw; Raw load(i,j,k,p)   loads forming u at an interior point
//   R form(const Raw&, i,j,k)       u from the loaded values
//   struct Ctr; Ctr load_ctr(p)     centre-only fields of the own point
//   void out(u, S, D, ctr, p, acc)  epilogue: S = sum c_q u_q, D = sum c_q
// plus the coefficient arrays kx, ky, kz of type Pol::TC.
#pragma once
#include "mg_device.cuh"

namespace mgdev {

constexpr int ZS_TX = 32, ZS_TY = 8, ZS_THREADS = ZS_TX * ZS_TY;

template <class Pol>
__global__ void __launch_bounds__(ZS_THREADS, 3) k_zs(Pol pol, Geom g, int kchunk, double* partials) {
  using R = typename Pol::R;
  using TC = typename Pol::TC;
  using Raw = typename Pol::Raw;
  using Ctr = typename Pol::Ctr;
  __shared__ R sp[3][ZS_TY + 2][ZS_TX + 2];
  pdl_wait();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i0 = blockIdx.x * ZS_TX, j0 = blockIdx.y * ZS_TY;
  const int i = i0 + lane, j = j0 + w;
  const int k0 = blockIdx.z * kchunk;
  const int k1 = min(k0 + kchunk, g.nz);
  const bool own_in_ij = i < g.nx && j < g.ny;
  const int sz = (int)g.sz;
  // halo points formed by this thread: warps 0 and 7 take the rows below and
  // above the tile, lanes 0 and 31 the columns left and right of their row
  const int hy_j = w == 0 ? j0 - 1 : (w == ZS_TY - 1 ? j0 + ZS_TY : -2);  // -2: none
  const int hx_i = lane == 0 ? i0 - 1 : (lane == 31 ? i0 + ZS_TX : -2);
  const bool has_hy = hy_j != -2 && i < g.nx && hy_j >= 0 && hy_j < g.ny;
  const bool has_hx = hx_i != -2 && j < g.ny && hx_i >= 0 && hx_i < g.nx;

  auto in_k = [&](int k) { return k >= 0 && k < g.nz; };
  // raw loads of plane k for the own point and the halo points (zero outside)
  struct Raws {
    Raw own, hy, hx;
  };
  auto load_plane = [&](int k, Raws& r) {
    const bool kin = in_k(k);
    if (own_in_ij && kin) r.own = pol.load(i, j, k, (int)g.at(i, j, k));
    if (has_hy && kin) r.hy = pol.load(i, hy_j, k, (int)g.at(i, hy_j, k));
    if (has_hx && kin) r.hx = pol.load(hx_i, j, k, (int)g.at(hx_i, j, k));
  };
  // forms u of plane k from the raws and stores it in shared plane s; returns the own value
  auto store_plane = [&](int k, const Raws& r, int s) -> R {
    const bool kin = in_k(k);
    const R uo = (own_in_ij && kin) ? pol.form(r.own, i, j, k) : (R)0;
    sp[s][w + 1][lane + 1] = uo;
    if (hy_j != -2) sp[s][w == 0 ? 0 : ZS_TY + 1][lane + 1] = (has_hy && kin) ? pol.form(r.hy, i, hy_j, k) : (R)0;
    if (hx_i != -2) sp[s][w + 1][lane == 0 ? 0 : ZS_TX + 1] = (has_hx && kin) ? pol.form(r.hx, hx_i, j, k) : (R)0;
    return uo;
  };

  double acc = 0.0, acc1 = 0.0;
  // prologue: u(k0-1) (own only), u(k0) into shared plane, raws of k0+1, centre fields of k0
  Raws rw{};
  R u_m = 0, u_c, u_p;
  {
    Raws r0{};
    if (own_in_ij && in_k(k0 - 1)) {
      r0.own = pol.load(i, j, k0 - 1, (int)g.at(i, j, k0 - 1));
      u_m = pol.form(r0.own, i, j, k0 - 1);
    }
  }
  {
    Raws r1{};
    load_plane(k0, r1);
    u_c = store_plane(k0, r1, k0 % 3);
  }
  load_plane(k0 + 1, rw);
  Ctr cn{};
  R kz_m = 0, kn_z = 0, kn_x = 0, kn_y = 0, kn_ym = 0, kn_xm = 0;
  auto load_coef = [&](int p, R& cx, R& cxm, R& cy, R& cym, R& cz) {
    cx = cvt<R>(__ldg(pol.kx + p));
    cxm = cvt<R>(__ldg(pol.kx + p - 1));
    cy = cvt<R>(__ldg(pol.ky + p));
    cym = cvt<R>(__ldg(pol.ky + p - g.Px));
    cz = cvt<R>(__ldg(pol.kz + p));
  };
  if (own_in_ij) {
    const int p0 = (int)g.at(i, j, k0);
    kz_m = cvt<R>(__ldg(pol.kz + p0 - sz));
    load_coef(p0, kn_x, kn_xm, kn_y, kn_ym, kn_z);
    cn = pol.load_ctr(p0);
  }
  for (int k = k0; k < k1; ++k) {
    // current-plane centre fields and coefficients (loaded one step ahead)
    const Ctr cc = cn;
    const R cxp = kn_x, cxm = kn_xm, cyp = kn_y, cym = kn_ym, czp = kn_z;
    // u of plane k+1 into shared memory
    u_p = store_plane(k + 1, rw, (k + 1) % 3);
    // loads for the next step: raws of plane k+2, centre fields of plane k+1
    if (k + 1 < k1) {
      load_plane(k + 2, rw);
      if (own_in_ij) {
        const int pn = (int)g.at(i, j, k + 1);
        load_coef(pn, kn_x, kn_xm, kn_y, kn_ym, kn_z);
        cn = pol.load_ctr(pn);
      }
    }
    __syncthreads();
    if (own_in_ij) {
      const int p = (int)g.at(i, j, k);
      const R(*P)[ZS_TX + 2] = sp[k % 3];
      R S = cxm * P[w + 1][lane];
      S = fma(cxp, P[w + 1][lane + 2], S);
      S = fma(cym, P[w][lane + 1], S);
      S = fma(cyp, P[w + 2][lane + 1], S);
      S = fma(kz_m, u_m, S);
      S = fma(czp, u_p, S);
      const R D = ((cxm + cxp) + (cym + cyp)) + (kz_m + czp);
      pol.out(u_c, S, D, cc, p, acc);
    }
    u_m = u_c;
    u_c = u_p;
    kz_m = czp;
  }
  pdl_trigger();
  if constexpr (Pol::kDot) {
    block_sum2<ZS_THREADS>(acc, acc1);
    if (threadIdx.x == 0) partials[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = acc;
  }
}

// ---- policies -----------------------------------------------------------------

// Chebyshev step j with materialised iterate (x_j -> x_{j+1}, d_j); kDot fuses
// rho = r.z (r float64) for the outer CG into the last step.
template <class R_, class TV, class TC_, bool kDot_> struct PolStep {
  using R = R_;
  using TC = TC_;
  static constexpr bool kDot = kDot_;
  const TV* x;
  const TV* dprev;
  const TV* b;
  const TV* dinv;
  TV* xout;
  TV* dout;
  const TC *kx, *ky, *kz;
  const double* r64;
  R c1, c2, inv_theta;
  struct Raw {
    TV x;
  };
  struct Ctr {
    TV b, dinv, d;
    double r;
  };
  __device__ __forceinline__ Raw load(int, int, int, int p) const { return {__ldg(x + p)}; }
  __device__ __forceinline__ R form(const Raw& r, int, int, int) const { return cvt<R>(r.x); }
  __device__ __forceinline__ Ctr load_ctr(int p) const {
    Ctr c;
    c.b = __ldg(b + p);
    c.dinv = sizeof(R) == 4 ? store_as<TV>(0.0) : __ldg(dinv + p);
    c.d = dprev ? __ldg(dprev + p) : store_as<TV>(0.0);
    c.r = kDot ? __ldg(r64 + p) : 0.0;
    return c;
  }
  __device__ __forceinline__ void out(R u, R S, R D, const Ctr& c, int p, double& acc) const {
    const R dv = sizeof(R) == 4 ? (R)1 / D : cvt<R>(c.dinv);
    const R s = fma(dv, cvt<R>(c.b) + S, -u);
    const R dn = dprev ? fma(c1, cvt<R>(c.d), c2 * s) : s * inv_theta;
    const TV xn = store_as<TV>(u + dn);
    xout[p] = xn;
    if (dout) dout[p] = store_as<TV>(dn);
    if constexpr (kDot) acc = fma(c.r, to_double(xn), acc);
  }
};

// First post-smoothing step with the coarse-grid correction folded in:
// u = x + P e (trilinear, formed per point), then step 0 of the sweep.
template <class R_, class TV, class TC_> struct PolProlongStep0 {
  using R = R_;
  using TC = TC_;
  static constexpr bool kDot = false;
  Geom gc;
  const TV* x;
  const TV* e;
  const TV* b;
  const TV* dinv;
  TV* xout;
  TV* dout;
  const TC *kx, *ky, *kz;
  R inv_theta;
  struct Raw {
    TV x, e[8];
  };
  struct Ctr {
    TV b, dinv;
  };
  __device__ __forceinline__ Raw load(int i, int j, int k, int p) const {
    Raw r;
    r.x = __ldg(x + p);
    const int ia = (i - 1) >> 1, jb = (j - 1) >> 1, kc = (k - 1) >> 1;
    const int di = (i >> 1) - ia, dj = ((j >> 1) - jb) * gc.Px, dk = ((k >> 1) - kc) * (int)gc.sz;
    const int q = (int)gc.at(ia, jb, kc);
    r.e[0] = __ldg(e + q);
    r.e[1] = __ldg(e + q + di);
    r.e[2] = __ldg(e + q + dj);
    r.e[3] = __ldg(e + q + dj + di);
    r.e[4] = __ldg(e + q + dk);
    r.e[5] = __ldg(e + q + dk + di);
    r.e[6] = __ldg(e + q + dk + dj);
    r.e[7] = __ldg(e + q + dk + dj + di);
    return r;
  }
  __device__ __forceinline__ R form(const Raw& r, int, int, int) const {
    R s = cvt<R>(r.e[0]) + cvt<R>(r.e[1]);
    s += cvt<R>(r.e[2]) + cvt<R>(r.e[3]);
    s += cvt<R>(r.e[4]) + cvt<R>(r.e[5]);
    s += cvt<R>(r.e[6]) + cvt<R>(r.e[7]);
    return fma((R)0.125, s, cvt<R>(r.x));
  }
  __device__ __forceinline__ Ctr load_ctr(int p) const {
    return {__ldg(b + p), sizeof(R) == 4 ? store_as<TV>(0.0) : __ldg(dinv + p)};
  }
  __device__ __forceinline__ void out(R u, R S, R D, const Ctr& c, int p, double&) const {
    const R dv = sizeof(R) == 4 ? (R)1 / D : cvt<R>(c.dinv);
    const R s = fma(dv, cvt<R>(c.b) + S, -u);
    const R dn = s * inv_theta;
    xout[p] = store_as<TV>(u + dn);
    if (dout) dout[p] = store_as<TV>(dn);
  }
};

// Steps 0 and 1 from a zero guess: u = x_1 = D^-1 b / theta.
template <class R_, class TV, class TC_> struct PolZero {
  using R = R_;
  using TC = TC_;
  static constexpr bool kDot = false;
  const TV* b;
  const TV* dinv;
  TV* xout;
  TV* dout;
  const TC *kx, *ky, *kz;
  R c1, c2, inv_theta;
  struct Raw {
    TV b, dinv;
  };
  struct Ctr {
    TV b, dinv;
  };
  __device__ __forceinline__ Raw load(int, int, int, int p) const { return {__ldg(b + p), __ldg(dinv + p)}; }
  __device__ __forceinline__ R form(const Raw& r, int, int, int) const {
    return inv_theta * (cvt<R>(r.dinv) * cvt<R>(r.b));
  }
  __device__ __forceinline__ Ctr load_ctr(int p) const { return {__ldg(b + p), __ldg(dinv + p)}; }
  __device__ __forceinline__ void out(R u, R S, R, const Ctr& c, int p, double&) const {
    const R s = fma(cvt<R>(c.dinv), cvt<R>(c.b) + S, -u);
    const R d1 = fma(c1, u, c2 * s);
    xout[p] = store_as<TV>(u + d1);
    if (dout) dout[p] = store_as<TV>(d1);
  }
};

// r = b - A x
template <class R_, class TV, class TC_> struct PolResid {
  using R = R_;
  using TC = TC_;
  static constexpr bool kDot = false;
  const TV* x;
  const TV* b;
  TV* r;
  const TC *kx, *ky, *kz;
  struct Raw {
    TV x;
  };
  struct Ctr {
    TV b;
  };
  __device__ __forceinline__ Raw load(int, int, int, int p) const { return {__ldg(x + p)}; }
  __device__ __forceinline__ R form(const Raw& rr, int, int, int) const { return cvt<R>(rr.x); }
  __device__ __forceinline__ Ctr load_ctr(int p) const { return {__ldg(b + p)}; }
  __device__ __forceinline__ void out(R u, R S, R D, const Ctr& c, int p, double&) const {
    r[p] = store_as<TV>((cvt<R>(c.b) + S) - D * u);
  }
};

}  // namespace mgdev
