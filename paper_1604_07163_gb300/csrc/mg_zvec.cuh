// Vectorised z-marching driver for the stencil passes (default kernel).
//
// Each thread owns two consecutive x points of a (2*32) x 4 tile and walks a
// chunk of planes.  Compared with one point per thread and all neighbours read
// through L1, three things keep more HBM bytes in flight per SM:
//   - the two points are read with one 8-byte (16-byte for float64) load per
//     array, and the x neighbours come from the adjacent lanes by warp
//     shuffles (only lanes 0 and 31 load theirs);
//   - the operand's z neighbours live in a register queue (planes k-1, k, k+1),
//     and everything read pointwise is loaded one plane ahead of its use;
//   - every streamed array is prefetched into L2 two planes ahead.
// The arithmetic is that of stencil() and the per-point operations in
// mg_device.cuh, term for term and in the same order, so results are
// bitwise identical to the one-point-per-thread kernel (only the block sums
// of the reducing passes group terms differently).
#pragma once
#include <type_traits>

#include "mg_device.cuh"

namespace mgdev {

constexpr int ZV_THREADS = 128;
constexpr int ZV_TX = 64, ZV_TY = 4;  // tile: 32 lanes x 2 points, 4 rows
constexpr int ZV_PF = 2;              // L2 prefetch distance in planes

// Two consecutive elements at a (a's index is even, so the vector access is
// aligned), converted to R.
template <class R> __device__ __forceinline__ void ld2(const float* a, R (&v)[2]) {
  const float2 t = __ldg(reinterpret_cast<const float2*>(a));
  v[0] = cvt<R>(t.x);
  v[1] = cvt<R>(t.y);
}
template <class R> __device__ __forceinline__ void ld2(const double* a, R (&v)[2]) {
  const double2 t = __ldg(reinterpret_cast<const double2*>(a));
  v[0] = cvt<R>(t.x);
  v[1] = cvt<R>(t.y);
}
template <class R> __device__ __forceinline__ void ld2(const __nv_bfloat16* a, R (&v)[2]) {
  const __nv_bfloat162 t = __ldg(reinterpret_cast<const __nv_bfloat162*>(a));
  v[0] = cvt<R>(t.x);
  v[1] = cvt<R>(t.y);
}
// Stores the first n (0, 1 or 2) of two consecutive results.
template <class R> __device__ __forceinline__ void st2(float* a, const R (&v)[2], int n) {
  if (n == 2) *reinterpret_cast<float2*>(a) = make_float2(store_as<float>(v[0]), store_as<float>(v[1]));
  else if (n == 1) a[0] = store_as<float>(v[0]);
}
template <class R> __device__ __forceinline__ void st2(double* a, const R (&v)[2], int n) {
  if (n == 2) *reinterpret_cast<double2*>(a) = make_double2(store_as<double>(v[0]), store_as<double>(v[1]));
  else if (n == 1) a[0] = store_as<double>(v[0]);
}
__device__ __forceinline__ void pf_l2(const void* a) { asm volatile("prefetch.global.L2 [%0];" ::"l"(a)); }

// Stencil neighbourhood of the two points p, p+1: operand values u and edge
// coefficients (c_x of the edge entering point 0 comes from the left lane).
template <class R> struct ZvNb {
  R uw, ue, cxw;
  R uc[2], um[2], up[2], us[2], un[2];
  R cx[2], cys[2], cy[2], czm[2], cz[2];
  // S and D of stencil() for element e
  __device__ __forceinline__ R eval(int e, R& D) const {
    const R cxm = e == 0 ? cxw : cx[0];
    const R xw = e == 0 ? uw : uc[0];
    const R xe = e == 1 ? ue : uc[1];
    D = ((cxm + cx[e]) + (cys[e] + cy[e])) + (czm[e] + cz[e]);
    R S = cxm * xw;
    S = fma(cx[e], xe, S);
    S = fma(cys[e], us[e], S);
    S = fma(cy[e], un[e], S);
    S = fma(czm[e], um[e], S);
    S = fma(cz[e], up[e], S);
    return S;
  }
};

// Per-operation hooks.  ok = false keeps an operation on the scalar driver.
//   U      operand storage of two points (what the stencil is applied to)
//   P      values read pointwise at the two points of the current plane
//   load_u / vals / u_one   operand of two points / as values / of one point
//   load_p                  pointwise values of a plane
//   prefetch(qp, qu)        L2 prefetch of the pointwise arrays at qp and of
//                           the operand arrays at qu
//   emit                    the point operation for the first nv points
template <class Op> struct Zv {
  static constexpr bool ok = false;
};

template <class R, class TV> struct ZvVecU {
  struct U {
    R v[2];
  };
  static __device__ __forceinline__ void load(const TV* a, int p, U& u) { ld2(a + p, u.v); }
  static __device__ __forceinline__ void vals(const U& u, R (&v)[2]) {
    v[0] = u.v[0];
    v[1] = u.v[1];
  }
  static __device__ __forceinline__ R one(const TV* a, int q) { return cvt<R>(__ldg(a + q)); }
};

// y = A u
template <class R_, class TV, class TC_> struct Zv<OpApply<R_, TV, TC_>> {
  using Op = OpApply<R_, TV, TC_>;
  using R = R_;
  using TC = TC_;
  using UU = ZvVecU<R, TV>;
  using U = typename UU::U;
  struct P {};
  static constexpr bool ok = true;
  static __device__ __forceinline__ const TC* kx(const Op& o) { return o.kx; }
  static __device__ __forceinline__ const TC* ky(const Op& o) { return o.ky; }
  static __device__ __forceinline__ const TC* kz(const Op& o) { return o.kz; }
  static __device__ __forceinline__ void load_u(const Op& o, int p, U& u) { UU::load(o.u, p, u); }
  static __device__ __forceinline__ void vals(const Op&, const U& u, R (&v)[2]) { UU::vals(u, v); }
  static __device__ __forceinline__ R u_one(const Op& o, int q) { return UU::one(o.u, q); }
  static __device__ __forceinline__ void load_p(const Op&, int, P&) {}
  static __device__ __forceinline__ void prefetch(const Op& o, int, int qu) { pf_l2(o.u + qu); }
  static __device__ __forceinline__ void emit(const Op& o, int p, int nv, const ZvNb<R>& nb, const U&, const P&,
                                              double&, double&) {
    R y[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      R D;
      const R S = nb.eval(e, D);
      y[e] = D * nb.uc[e] - S;
    }
    st2(o.y + p, y, nv);
  }
};

// Chebyshev step (OpChebStep): the pointwise part shared with the fused dot.
template <class R, class TV, class TC> struct ZvStepP {
  R b[2], d[2], di[2];
};
template <class R, class TV, class TC>
__device__ __forceinline__ void zv_step_load_p(const OpChebStep<R, TV, TC>& o, int p, ZvStepP<R, TV, TC>& P) {
  ld2(o.b + p, P.b);
  if (o.dprev) ld2(o.dprev + p, P.d);
  if constexpr (sizeof(R) == 8) ld2(o.dinv + p, P.di);
}
template <class R, class TV, class TC>
__device__ __forceinline__ void zv_step_prefetch(const OpChebStep<R, TV, TC>& o, int qp, int qu) {
  pf_l2(o.x + qu);
  pf_l2(o.b + qp);
  if (o.dprev) pf_l2(o.dprev + qp);
  if constexpr (sizeof(R) == 8) pf_l2(o.dinv + qp);
}
// x_{j+1} of the two points, stored; returns them in xn
template <class R, class TV, class TC>
__device__ __forceinline__ void zv_step_emit(const OpChebStep<R, TV, TC>& o, int p, int nv, const ZvNb<R>& nb,
                                             const ZvStepP<R, TV, TC>& P, R (&xn)[2]) {
  R dn[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    R D;
    const R S = nb.eval(e, D);
    const R xp = nb.uc[e];
    R inv;
    if constexpr (sizeof(R) == 4) inv = (R)1 / D;
    else inv = P.di[e];
    const R s = fma(inv, P.b[e] + S, -xp);
    dn[e] = o.dprev ? fma(o.c1, P.d[e], o.c2 * s) : s * o.inv_theta;
    xn[e] = xp + dn[e];
  }
  st2(o.xout + p, xn, nv);
  if (o.dout) st2(o.dout + p, dn, nv);
}

template <class R_, class TV, class TC_> struct Zv<OpChebStep<R_, TV, TC_>> {
  using Op = OpChebStep<R_, TV, TC_>;
  using R = R_;
  using TC = TC_;
  using UU = ZvVecU<R, TV>;
  using U = typename UU::U;
  using P = ZvStepP<R, TV, TC>;
  static constexpr bool ok = true;
  static __device__ __forceinline__ const TC* kx(const Op& o) { return o.kx; }
  static __device__ __forceinline__ const TC* ky(const Op& o) { return o.ky; }
  static __device__ __forceinline__ const TC* kz(const Op& o) { return o.kz; }
  static __device__ __forceinline__ void load_u(const Op& o, int p, U& u) { UU::load(o.x, p, u); }
  static __device__ __forceinline__ void vals(const Op&, const U& u, R (&v)[2]) { UU::vals(u, v); }
  static __device__ __forceinline__ R u_one(const Op& o, int q) { return UU::one(o.x, q); }
  static __device__ __forceinline__ void load_p(const Op& o, int p, P& q) { zv_step_load_p(o, p, q); }
  static __device__ __forceinline__ void prefetch(const Op& o, int qp, int qu) { zv_step_prefetch(o, qp, qu); }
  static __device__ __forceinline__ void emit(const Op& o, int p, int nv, const ZvNb<R>& nb, const U&, const P& q,
                                              double&, double&) {
    R xn[2];
    zv_step_emit(o, p, nv, nb, q, xn);
  }
};

// Compensated dot-product step (Ogita, Rump and Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 2005, algorithm Dot2): adds x*y to the
// float-float accumulator (s, c).  x*y = h + r exactly (TwoProduct via FMA),
// s + h = t + q exactly (Knuth's TwoSum), and c collects q + r.  After n terms
// s + c is the dot product with error at most about (n u)^2 sum |x y|, u =
// 2^-24, i.e. as if summed in twice the float32 precision.  The __f*_rn
// intrinsics keep the compiler from contracting the product into the sums.
__device__ __forceinline__ void dot2_add(float x, float y, float& s, float& c) {
  const float h = __fmul_rn(x, y);
  const float r = fmaf(x, y, -h);
  const float t = __fadd_rn(s, h);
  const float bp = __fsub_rn(t, s);
  const float q = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(h, bp));
  s = t;
  c = __fadd_rn(c, __fadd_rn(q, r));
}

// Ops whose Zv hooks define float_acc = true sum their per-point terms in a
// float-float pair per thread (emit_f), which the driver adds into the
// float64 block sum after its plane loop.
template <class Z, class = void> struct ZvFloatAcc : std::false_type {};
template <class Z>
struct ZvFloatAcc<Z, std::void_t<decltype(Z::float_acc)>> : std::integral_constant<bool, Z::float_acc> {};

// last post-smoothing step with rho = b.z accumulated (OpChebStepDot: b is
// the right-hand side the step already reads, held exactly in R).  float64
// form: one float64 FMA per point.  Float32 V-cycle forms: the products of
// the float32 b and z are summed per thread with dot2_add on the float32
// pipe, so the pass needs no widening and no float64 operation per point.
template <class R_, class TV, class TC_> struct Zv<OpChebStepDot<R_, TV, TC_>> {
  using Op = OpChebStepDot<R_, TV, TC_>;
  using R = R_;
  using TC = TC_;
  using UU = ZvVecU<R, TV>;
  using U = typename UU::U;
  using P = ZvStepP<R, TV, TC>;
  static constexpr bool ok = true;
  static __device__ __forceinline__ const TC* kx(const Op& o) { return o.step.kx; }
  static __device__ __forceinline__ const TC* ky(const Op& o) { return o.step.ky; }
  static __device__ __forceinline__ const TC* kz(const Op& o) { return o.step.kz; }
  static __device__ __forceinline__ void load_u(const Op& o, int p, U& u) { UU::load(o.step.x, p, u); }
  static __device__ __forceinline__ void vals(const Op&, const U& u, R (&v)[2]) { UU::vals(u, v); }
  static __device__ __forceinline__ R u_one(const Op& o, int q) { return UU::one(o.step.x, q); }
  static __device__ __forceinline__ void load_p(const Op& o, int p, P& q) { zv_step_load_p(o.step, p, q); }
  static __device__ __forceinline__ void prefetch(const Op& o, int qp, int qu) { zv_step_prefetch(o.step, qp, qu); }
  static constexpr bool float_acc = sizeof(R) == 4 && sizeof(TV) == 4;
  static __device__ __forceinline__ void emit(const Op& o, int p, int nv, const ZvNb<R>& nb, const U&, const P& q,
                                              double& a0, double&) {
    R xn[2];
    zv_step_emit(o.step, p, nv, nb, q, xn);
    if (nv > 0) a0 = fma(to_double(store_as<TV>(q.b[0])), to_double(store_as<TV>(xn[0])), a0);
    if (nv > 1) a0 = fma(to_double(store_as<TV>(q.b[1])), to_double(store_as<TV>(xn[1])), a0);
  }
  static __device__ __forceinline__ void emit_f(const Op& o, int p, int nv, const ZvNb<R>& nb, const U&,
                                                const P& q, float& s, float& c) {
    R xn[2];
    zv_step_emit(o.step, p, nv, nb, q, xn);
    if (nv > 0) dot2_add((float)q.b[0], (float)store_as<TV>(xn[0]), s, c);
    if (nv > 1) dot2_add((float)q.b[1], (float)store_as<TV>(xn[1]), s, c);
  }
};

// pre-smoothing from a zero guess: the operand x_1 = D^-1 b / theta is formed
// from b and D^-1 at every stencil point
template <class R_, class TV, class TC_> struct Zv<OpChebZero<R_, TV, TC_>> {
  using Op = OpChebZero<R_, TV, TC_>;
  using R = R_;
  using TC = TC_;
  struct U {
    R b[2], di[2];
  };
  struct P {};
  static constexpr bool ok = true;
  static __device__ __forceinline__ const TC* kx(const Op& o) { return o.kx; }
  static __device__ __forceinline__ const TC* ky(const Op& o) { return o.ky; }
  static __device__ __forceinline__ const TC* kz(const Op& o) { return o.kz; }
  static __device__ __forceinline__ void load_u(const Op& o, int p, U& u) {
    ld2(o.b + p, u.b);
    ld2(o.dinv + p, u.di);
  }
  static __device__ __forceinline__ void vals(const Op& o, const U& u, R (&v)[2]) {
    v[0] = o.inv_theta * (u.di[0] * u.b[0]);
    v[1] = o.inv_theta * (u.di[1] * u.b[1]);
  }
  static __device__ __forceinline__ R u_one(const Op& o, int q) {
    return o.inv_theta * (cvt<R>(__ldg(o.dinv + q)) * cvt<R>(__ldg(o.b + q)));
  }
  static __device__ __forceinline__ void load_p(const Op&, int, P&) {}
  static __device__ __forceinline__ void prefetch(const Op& o, int, int qu) {
    pf_l2(o.b + qu);
    pf_l2(o.dinv + qu);
  }
  static __device__ __forceinline__ void emit(const Op& o, int p, int nv, const ZvNb<R>& nb, const U& uc, const P&,
                                              double&, double&) {
    R xo[2], d1[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      R D;
      const R S = nb.eval(e, D);
      const R x1 = nb.uc[e];
      const R s = fma(uc.di[e], uc.b[e] + S, -x1);
      d1[e] = fma(o.c1, x1, o.c2 * s);
      xo[e] = x1 + d1[e];
    }
    st2(o.xout + p, xo, nv);
    if (o.dout) st2(o.dout + p, d1, nv);
  }
};

// r = b - A x (acc0 += r.r)
template <class R_, class TV, class TB, class TC_> struct Zv<OpResidual<R_, TV, TB, TC_>> {
  using Op = OpResidual<R_, TV, TB, TC_>;
  using R = R_;
  using TC = TC_;
  using UU = ZvVecU<R, TV>;
  using U = typename UU::U;
  struct P {
    R b[2];
  };
  static constexpr bool ok = true;
  static __device__ __forceinline__ const TC* kx(const Op& o) { return o.kx; }
  static __device__ __forceinline__ const TC* ky(const Op& o) { return o.ky; }
  static __device__ __forceinline__ const TC* kz(const Op& o) { return o.kz; }
  static __device__ __forceinline__ void load_u(const Op& o, int p, U& u) { UU::load(o.x, p, u); }
  static __device__ __forceinline__ void vals(const Op&, const U& u, R (&v)[2]) { UU::vals(u, v); }
  static __device__ __forceinline__ R u_one(const Op& o, int q) { return UU::one(o.x, q); }
  static __device__ __forceinline__ void load_p(const Op& o, int p, P& q) { ld2(o.b + p, q.b); }
  static __device__ __forceinline__ void prefetch(const Op& o, int qp, int qu) {
    pf_l2(o.x + qu);
    pf_l2(o.b + qp);
  }
  static __device__ __forceinline__ void emit(const Op& o, int p, int nv, const ZvNb<R>& nb, const U&, const P& q,
                                              double& acc, double&) {
    R rv[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      R D;
      const R S = nb.eval(e, D);
      rv[e] = (q.b[e] + S) - D * nb.uc[e];
    }
    st2(o.r + p, rv, nv);
    if (nv > 0) acc = fma((double)rv[0], (double)rv[0], acc);
    if (nv > 1) acc = fma((double)rv[1], (double)rv[1], acc);
  }
};

// float64 r = b - A x with the stored diagonal
template <class TB> struct Zv<OpResidualD<TB>> {
  using Op = OpResidualD<TB>;
  using R = double;
  using TC = double;
  using UU = ZvVecU<double, double>;
  using U = typename UU::U;
  struct P {
    double b[2], dg[2];
  };
  static constexpr bool ok = true;
  static __device__ __forceinline__ const TC* kx(const Op& o) { return o.kx; }
  static __device__ __forceinline__ const TC* ky(const Op& o) { return o.ky; }
  static __device__ __forceinline__ const TC* kz(const Op& o) { return o.kz; }
  static __device__ __forceinline__ void load_u(const Op& o, int p, U& u) { UU::load(o.x, p, u); }
  static __device__ __forceinline__ void vals(const Op&, const U& u, double (&v)[2]) { UU::vals(u, v); }
  static __device__ __forceinline__ double u_one(const Op& o, int q) { return UU::one(o.x, q); }
  static __device__ __forceinline__ void load_p(const Op& o, int p, P& q) {
    ld2(o.b + p, q.b);
    ld2(o.dg + p, q.dg);
  }
  static __device__ __forceinline__ void prefetch(const Op& o, int qp, int qu) {
    pf_l2(o.x + qu);
    pf_l2(o.b + qp);
    pf_l2(o.dg + qp);
  }
  static __device__ __forceinline__ void emit(const Op& o, int p, int nv, const ZvNb<double>& nb, const U&, const P& q,
                                              double& acc, double&) {
    double rv[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      double D;
      const double S = nb.eval(e, D);
      rv[e] = (q.b[e] + S) - q.dg[e] * nb.uc[e];
    }
    st2(o.r + p, rv, nv);
    if (nv > 0) acc = fma(rv[0], rv[0], acc);
    if (nv > 1) acc = fma(rv[1], rv[1], acc);
  }
};

// (The float64 CG operator, OpApplyPQ, stays on the scalar driver: it is bound
// by the float64 pipe, and the scalar kernel measured 3% faster on it.)

// Resident blocks per SM requested from the compiler: 8 (64 registers per
// thread) for float32 arithmetic, 4 for float64.
template <class Op> struct ZvMinBlocks {
  static constexpr int value = sizeof(typename Zv<Op>::R) == 8 ? 4 : 8;
};

// The driver.  Rows j >= ny are whole warps and skip the loop (they still take
// part in the block sum); lanes past the padded row read their own row's pad
// slots and store nothing, so every shuffle has all 32 lanes.
template <class Op, bool RED>
__global__ void __launch_bounds__(ZV_THREADS, ZvMinBlocks<Op>::value)
    k_zvec(Op op, Geom g, int kchunk, double* partials, int stride) {
  using Z = Zv<Op>;
  using R = typename Z::R;
  using TC = typename Z::TC;
  using U = typename Z::U;
  using P = typename Z::P;
  pdl_wait();
  op.prepare();
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * ZV_TX + 2 * lane;
  const int j = blockIdx.y * ZV_TY + (threadIdx.x >> 5);
  const int k0 = blockIdx.z * kchunk;
  const int k1 = min(k0 + kchunk, g.nz);
  double a0 = 0.0, a1 = 0.0;
  float f0 = 0.0f, f1 = 0.0f;  // float-float accumulator (ZvFloatAcc ops)
  if (j < g.ny) {
    const int nv = min(max(g.nx - i, 0), 2);
    const int sz = (int)g.sz, sy = g.Px;
    int p = (int)g.at(min(i, g.Px - 2), j, k0);
    const TC* kx = Z::kx(op);
    const TC* ky = Z::ky(op);
    const TC* kz = Z::kz(op);
    U qm, qc, qp;
    Z::load_u(op, p - sz, qm);
    Z::load_u(op, p, qc);
    Z::load_u(op, p + sz, qp);
    R czm[2], nkx[2], nky[2], nkz[2];
    ld2(kz + p - sz, czm);
    ld2(kx + p, nkx);
    ld2(ky + p, nky);
    ld2(kz + p, nkz);
    P pn;
    Z::load_p(op, p, pn);
    for (int k = k0; k < k1; ++k, p += sz) {
      ZvNb<R> nb;
      const P pc = pn;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        nb.cx[e] = nkx[e];
        nb.cy[e] = nky[e];
        nb.cz[e] = nkz[e];
        nb.czm[e] = czm[e];
      }
      U qn = qp;
      if (k + 1 < k1) {  // next plane: operand two planes up, pointwise values one plane up
        Z::load_u(op, p + 2 * sz, qn);
        Z::load_p(op, p + sz, pn);
        ld2(kx + p + sz, nkx);
        ld2(ky + p + sz, nky);
        ld2(kz + p + sz, nkz);
      }
      if (k + ZV_PF < k1) {
        const int q = p + ZV_PF * sz;
        pf_l2(kx + q);
        pf_l2(ky + q);
        pf_l2(kz + q);
        Z::prefetch(op, q, q + sz);
      }
      U ys, yn;
      Z::load_u(op, p - sy, ys);
      Z::load_u(op, p + sy, yn);
      ld2(ky + p - sy, nb.cys);
      Z::vals(op, qc, nb.uc);
      Z::vals(op, qm, nb.um);
      Z::vals(op, qp, nb.up);
      Z::vals(op, ys, nb.us);
      Z::vals(op, yn, nb.un);
      nb.uw = __shfl_up_sync(0xffffffffu, nb.uc[1], 1);
      nb.ue = __shfl_down_sync(0xffffffffu, nb.uc[0], 1);
      nb.cxw = __shfl_up_sync(0xffffffffu, nb.cx[1], 1);
      if (lane == 0) {
        nb.uw = Z::u_one(op, p - 1);
        nb.cxw = cvt<R>(__ldg(kx + p - 1));
      }
      if (lane == 31) nb.ue = Z::u_one(op, p + 2);
      if (nv > 0) {
        if constexpr (ZvFloatAcc<Z>::value) Z::emit_f(op, p, nv, nb, qc, pc, f0, f1);
        else Z::emit(op, p, nv, nb, qc, pc, a0, a1);
      }
      qm = qc;
      qc = qp;
      qp = qn;
#pragma unroll
      for (int e = 0; e < 2; ++e) czm[e] = nb.cz[e];
    }
  }
  pdl_trigger();
  if constexpr (RED) {
    if constexpr (ZvFloatAcc<Z>::value) a0 = (double)f0 + (double)f1;  // exact widening, once per thread
    block_sum2<ZV_THREADS>(a0, a1);
    if (threadIdx.x == 0) {
      const int b = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      partials[b] = a0;
      partials[stride + b] = a1;
    }
  }
}

// ------------------------------------------------------------ transfers
// x += P e on the fine grid (OpProlong) without z-marching: each thread
// updates four consecutive fine points of one row (one 16-byte access to x in
// float32, two in float64); the twelve coarse values they draw on (coarse
// columns 2m-1 .. 2m+1, two rows, two planes) come through L1.  A thread
// owns one row chunk, so many independent read-modify-writes are in flight.
// Same terms in the same order as OpProlong; each coarse column's sum is
// formed once for the four points.
constexpr int PV_THREADS = 256;  // 64 chunks of 4 points x 4 rows
template <class R, class TV>
__global__ void __launch_bounds__(PV_THREADS) k_prolong_v(OpProlong<R, TV> op, Geom g) {
  pdl_wait();
  const int chunk = blockIdx.x * 64 + (threadIdx.x & 63);
  const int j = blockIdx.y * 4 + (threadIdx.x >> 6);
  const int k = blockIdx.z;
  const int i = 4 * chunk;
  if (j < g.ny && i < g.nx) {
    const Geom& gc = op.gc;
    const int m = chunk;  // fine i = 4m: coarse columns 2m-1, 2m, 2m+1
    const int jr[2] = {(j - 1) >> 1, j >> 1}, kp[2] = {(k - 1) >> 1, k >> 1};
    R E[2][2][3];  // [plane k0/k1][row j0/j1][column 2m-1 .. 2m+1]
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const i64 q = gc.at(2 * m - 1, jr[r], kp[a]);
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) E[a][r][cc] = cvt<R>(__ldg(op.e + q + cc));
      }
    const i64 p = g.at(i, j, k);
    R xv[4];
    if constexpr (sizeof(TV) == 4) {
      const float4 t = *reinterpret_cast<const float4*>(op.x + p);
      xv[0] = t.x, xv[1] = t.y, xv[2] = t.z, xv[3] = t.w;
    } else {
      const double2 t0 = *reinterpret_cast<const double2*>(op.x + p);
      const double2 t1 = *reinterpret_cast<const double2*>(op.x + p + 2);
      xv[0] = t0.x, xv[1] = t0.y, xv[2] = t1.x, xv[3] = t1.y;
    }
    R Y[3];  // per coarse column: the two rows and two planes, in OpProlong's order
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) Y[cc] = (E[0][0][cc] + E[1][0][cc]) + (E[0][1][cc] + E[1][1][cc]);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      // coarse columns of fine 4m+e: i0 = (4m+e-1)>>1, i1 = (4m+e)>>1, as offsets from 2m-1
      const int c0 = (e + 1) >> 1, c1 = (e + 2) >> 1;
      xv[e] = fma((R)0.125, Y[c0] + Y[c1], xv[e]);
    }
    const int nv = min(g.nx - i, 4);
    if (nv == 4) {
      if constexpr (sizeof(TV) == 4) {
        *reinterpret_cast<float4*>(op.x + p) = make_float4(xv[0], xv[1], xv[2], xv[3]);
      } else {
        reinterpret_cast<double2*>(op.x + p)[0] = make_double2(xv[0], xv[1]);
        reinterpret_cast<double2*>(op.x + p)[1] = make_double2(xv[2], xv[3]);
      }
    } else {
      for (int e = 0; e < nv; ++e) op.x[p + e] = store_as<TV>(xv[e]);
    }
  }
  pdl_trigger();
}

// bc = R r on the coarse grid (OpRestrict), two coarse points (c, c+1) per
// thread: the five fine values 2c .. 2c+4 of a fine row come from one
// 16-byte load and the right lane's first value.  Per fine plane the three
// fine rows give the plane sum; consecutive coarse planes share a fine plane,
// whose sum is kept.  Same terms in the same order as OpRestrict.
template <class R, class TV>
__global__ void __launch_bounds__(ZV_THREADS, 8) k_restrict_v(OpRestrict<R, TV> op, Geom gc, int kchunk) {
  pdl_wait();
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * ZV_TX + 2 * lane;
  const int cj = blockIdx.y * ZV_TY + (threadIdx.x >> 5);
  const int k0 = blockIdx.z * kchunk;
  const int k1 = min(k0 + kchunk, gc.nz);
  if (cj < gc.ny) {
    const Geom& gf = op.gf;
    const int nv = min(max(gc.nx - c, 0), 2);
    const int fb = min(2 * c, gf.Px - 4);  // fine x of the first of the five values (a multiple of 4)
    // plane sum of fine plane kf for the two coarse points
    auto plane = [&](int kf, R (&P)[2]) {
      R row[3][2];
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const int q = (int)gf.at(fb, 2 * cj + b, kf);
        R v[5];
        if constexpr (sizeof(TV) == 4) {
          const float4 t = __ldg(reinterpret_cast<const float4*>(op.r + q));
          v[0] = cvt<R>(t.x), v[1] = cvt<R>(t.y), v[2] = cvt<R>(t.z), v[3] = cvt<R>(t.w);
        } else {
          const double2 t0 = __ldg(reinterpret_cast<const double2*>(op.r + q));
          const double2 t1 = __ldg(reinterpret_cast<const double2*>(op.r + q + 2));
          v[0] = cvt<R>(t0.x), v[1] = cvt<R>(t0.y), v[2] = cvt<R>(t1.x), v[3] = cvt<R>(t1.y);
        }
        v[4] = __shfl_down_sync(0xffffffffu, v[0], 1);
        if (lane == 31) v[4] = cvt<R>(__ldg(op.r + q + 4));
#pragma unroll
        for (int e = 0; e < 2; ++e)
          row[b][e] = fma((R)0.5, v[2 * e + 1], (R)0.25 * (v[2 * e] + v[2 * e + 2]));
      }
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        R pl = 0;
        pl = fma((R)0.25, row[0][e], pl);
        pl = fma((R)0.5, row[1][e], pl);
        pl = fma((R)0.25, row[2][e], pl);
        P[e] = pl;
      }
    };
    R Plo[2], Pmid[2], Phi[2];
    plane(2 * k0, Plo);
    for (int k = k0; k < k1; ++k) {
      if (k + 1 < k1) {  // the fine rows of the next coarse plane into L2
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          pf_l2(op.r + gf.at(fb, 2 * cj + b, 2 * k + 3));
          pf_l2(op.r + gf.at(fb, 2 * cj + b, 2 * k + 4));
        }
      }
      plane(2 * k + 1, Pmid);
      plane(2 * k + 2, Phi);
      R acc[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        R a = 0;
        a = fma((R)0.25, Plo[e], a);
        a = fma((R)0.5, Pmid[e], a);
        a = fma((R)0.25, Phi[e], a);
        acc[e] = a;
      }
      if (nv > 0) st2(op.bc + gc.at(min(c, gc.Px - 2), cj, k), acc, nv);
#pragma unroll
      for (int e = 0; e < 2; ++e) Plo[e] = Phi[e];
    }
  }
  pdl_trigger();
}

template <class Op> struct ZvXfer {
  static constexpr bool ok = false;
};
template <class R, class TV> struct ZvXfer<OpProlong<R, TV>> {
  static constexpr bool ok = true;
};
template <class R, class TV> struct ZvXfer<OpRestrict<R, TV>> {
  static constexpr bool ok = true;
};

}  // namespace mgdev
