// Device-side building blocks of the multigrid-preconditioned CG solve.
//
// Data layout (every level, every nodal array): only interior unknowns are
// stored, in a padded [z][y][x] layout whose pad slots are kept at zero.  Row
// pitch Px >= nx+1 (multiple of 8), Py = ny+1 rows per plane, one pad plane in
// front of plane 0 and one after plane nz-1.  Interior point (i,j,k) sits at
// off + (k*Py + j)*Px + i.  Every one of the 26 neighbours of an interior
// point then lands either on an interior point or on a zero pad slot, so the
// Dirichlet boundary (x = 0 there) needs no branches in the stencil, the
// restriction or the prolongation.
//
// Edge coefficients use the same layout: kx[at(i,j,k)] is h_x^-2 k_e of the
// edge from interior point (i,j,k) to (i+1,j,k); the edge entering point
// (0,j,k) from the boundary lives at at(-1,j,k), which is a pad slot of the
// x-row before.  ky and kz likewise.  The stencil of Eq. 2 at point p is then
//   (A u)_p = D_p u_p - S_p,   S_p = sum_q c_pq u_q,   D_p = sum_q c_pq
// with c_pq read from kx[p-1], kx[p], ky[p-Px], ky[p], kz[p-Px*Py], kz[p].
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mgdev {

typedef long long i64;

struct Geom {
  int nx, ny, nz;  // interior points per axis
  int Px, Py;      // elements per padded row, rows per plane
  i64 sz;          // elements per plane
  i64 off;         // index of interior point (0,0,0)
  i64 len;         // allocation length in elements
  __host__ __device__ __forceinline__ i64 at(int i, int j, int k) const {
    return off + ((i64)k * Py + j) * Px + i;
  }
  __host__ __device__ __forceinline__ i64 npts() const { return (i64)nx * ny * nz; }
};

// ------------------------------------------------------------ conversions
template <class R> __device__ __forceinline__ R cvt(double v) { return (R)v; }
template <class R> __device__ __forceinline__ R cvt(float v) { return (R)v; }
template <class R> __device__ __forceinline__ R cvt(__nv_bfloat16 v) { return (R)__bfloat162float(v); }

template <class T> __device__ __forceinline__ T store_as(double v) { return (T)v; }
template <class T> __device__ __forceinline__ T store_as(float v) { return (T)v; }
template <> __device__ __forceinline__ __nv_bfloat16 store_as<__nv_bfloat16>(double v) {
  return __double2bfloat16(v);
}
template <> __device__ __forceinline__ __nv_bfloat16 store_as<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}

// Loads: NC = true uses the read-only path (data not written by this kernel);
// NC = false is a plain coherent load (the single-block bottom kernel reads
// what its own threads wrote before a __syncthreads()).
template <bool NC, class T> __device__ __forceinline__ T ldp(const T* p) {
  if constexpr (NC) return __ldg(p);
  else return *p;
}

// ------------------------------------------------------------ loaders
template <bool NC, class R, class T> struct LdVec {
  const T* a;
  __device__ __forceinline__ R operator()(i64 q) const { return cvt<R>(ldp<NC>(a + q)); }
};
// First Chebyshev iterate from a zero guess: x_1 = D^-1 b / theta.
template <bool NC, class R, class TV> struct LdJac {
  const TV* b;
  const TV* dinv;
  R inv_theta;
  __device__ __forceinline__ R operator()(i64 q) const {
    return inv_theta * (cvt<R>(ldp<NC>(dinv + q)) * cvt<R>(ldp<NC>(b + q)));
  }
};
// CG search direction formed on the fly: p_new = z + beta p_old.
template <bool NC> struct LdDir {
  const double* z;
  const double* p;
  double beta;
  __device__ __forceinline__ double operator()(i64 q) const { return fma(beta, ldp<NC>(p + q), ldp<NC>(z + q)); }
};

// S_p = sum_q c_pq u_q and D_p = sum_q c_pq at interior point p.
template <bool NC, class R, class TC, class U>
__device__ __forceinline__ R stencil(const Geom& g, i64 p, const U& u, const TC* kx, const TC* ky, const TC* kz,
                                     R& D) {
  const i64 sy = g.Px, sz = g.sz;
  const R cxm = cvt<R>(ldp<NC>(kx + p - 1)), cxp = cvt<R>(ldp<NC>(kx + p));
  const R cym = cvt<R>(ldp<NC>(ky + p - sy)), cyp = cvt<R>(ldp<NC>(ky + p));
  const R czm = cvt<R>(ldp<NC>(kz + p - sz)), czp = cvt<R>(ldp<NC>(kz + p));
  D = ((cxm + cxp) + (cym + cyp)) + (czm + czp);
  R S = cxm * u(p - 1);
  S = fma(cxp, u(p + 1), S);
  S = fma(cym, u(p - sy), S);
  S = fma(cyp, u(p + sy), S);
  S = fma(czm, u(p - sz), S);
  S = fma(czp, u(p + sz), S);
  return S;
}

// ------------------------------------------------------------ point operations
// Every op exposes  template<bool NC> void pt(g, i, j, k, p, acc0, acc1)
// and  prepare()  (called once per thread before the point loop).

// y = A u
template <class R, class TV, class TC> struct OpApply {
  const TV* u;
  TV* y;
  const TC *kx, *ky, *kz;
  __device__ void prepare() {}
  template <bool NC> __device__ __forceinline__ void pt(const Geom& g, int, int, int, i64 p, double&, double&) const {
    R D;
    LdVec<NC, R, TV> lu{u};
    R S = stencil<NC, R>(g, p, lu, kx, ky, kz, D);
    y[p] = store_as<TV>(D * lu(p) - S);
  }
};

// Chebyshev iteration for D^-1 A (Saad, Iterative Methods, Alg. 12.1), one
// step j with materialised iterate x_j:
//   s_j = D^-1 (b - A x_j)  evaluated as  D^-1 (b + S) - x_j  (D^-1 D = 1)
//   d_j = s_j / theta (j = 0)  or  c1 d_{j-1} + c2 s_j,  x_{j+1} = x_j + d_j.
template <class R, class TV, class TC> struct OpChebStep {
  const TV* x;
  const TV* dprev;  // null for j = 0
  const TV* b;
  const TV* dinv;
  TV* xout;
  TV* dout;  // null when d_j is not needed afterwards
  const TC *kx, *ky, *kz;
  R c1, c2, inv_theta;
  __device__ void prepare() {}
  template <bool NC> __device__ __forceinline__ void pt(const Geom& g, int, int, int, i64 p, double&, double&) const {
    R D;
    LdVec<NC, R, TV> lx{x};
    R S = stencil<NC, R>(g, p, lx, kx, ky, kz, D);
    const R xp = lx(p);
    const R s = fma(cvt<R>(ldp<NC>(dinv + p)), cvt<R>(ldp<NC>(b + p)) + S, -xp);
    const R dn = dprev ? fma(c1, cvt<R>(ldp<NC>(dprev + p)), c2 * s) : s * inv_theta;
    xout[p] = store_as<TV>(xp + dn);
    if (dout) dout[p] = store_as<TV>(dn);
  }
};

// Steps 0 and 1 of a sweep from a zero initial guess in one pass:
//   x_1 = d_0 = D^-1 b / theta (formed on the fly at the 7 stencil points),
//   s_1 = D^-1 (b - A x_1), d_1 = c1 d_0 + c2 s_1, x_2 = x_1 + d_1.
template <class R, class TV, class TC> struct OpChebZero {
  const TV* b;
  const TV* dinv;
  TV* xout;
  TV* dout;
  const TC *kx, *ky, *kz;
  R c1, c2, inv_theta;
  __device__ void prepare() {}
  template <bool NC> __device__ __forceinline__ void pt(const Geom& g, int, int, int, i64 p, double&, double&) const {
    R D;
    LdJac<NC, R, TV> lx{b, dinv, inv_theta};
    R S = stencil<NC, R>(g, p, lx, kx, ky, kz, D);
    const R x1 = lx(p);
    const R s = fma(cvt<R>(ldp<NC>(dinv + p)), cvt<R>(ldp<NC>(b + p)) + S, -x1);
    const R d1 = fma(c1, x1, c2 * s);
    xout[p] = store_as<TV>(x1 + d1);
    if (dout) dout[p] = store_as<TV>(d1);
  }
};

// Degree-1 sweep from a zero guess: x_1 = D^-1 b / theta.
template <class R, class TV> struct OpChebZero1 {
  const TV* b;
  const TV* dinv;
  TV* xout;
  R inv_theta;
  __device__ void prepare() {}
  template <bool NC> __device__ __forceinline__ void pt(const Geom&, int, int, int, i64 p, double&, double&) const {
    xout[p] = store_as<TV>(inv_theta * (cvt<R>(ldp<NC>(dinv + p)) * cvt<R>(ldp<NC>(b + p))));
  }
};

// r = b - A x
template <class R, class TV, class TB, class TC> struct OpResidual {
  const TV* x;
  const TB* b;
  TV* r;
  const TC *kx, *ky, *kz;
  __device__ void prepare() {}
  template <bool NC> __device__ __forceinline__ void pt(const Geom& g, int, int, int, i64 p, double& acc,
                                                        double&) const {
    R D;
    LdVec<NC, R, TV> lx{x};
    R S = stencil<NC, R>(g, p, lx, kx, ky, kz, D);
    const R rv = (cvt<R>(ldp<NC>(b + p)) + S) - D * lx(p);
    r[p] = store_as<TV>(rv);
    acc = fma((double)rv, (double)rv, acc);
  }
};

// Full weighting bc = R r, R = P^T / 8: weights (1/4, 1/2, 1/4) per axis
// around fine point (2i+1, 2j+1, 2k+1), the image of coarse point (i,j,k).
// Runs over the coarse grid; gf is the fine geometry.
template <class R, class TV> struct OpRestrict {
  Geom gf;
  const TV* r;
  TV* bc;
  __device__ void prepare() {}
  template <bool NC> __device__ __forceinline__ void pt(const Geom&, int i, int j, int k, i64 pc, double&,
                                                        double&) const {
    const i64 pf = gf.at(2 * i + 1, 2 * j + 1, 2 * k + 1);
    R acc = 0;
#pragma unroll
    for (int c = -1; c <= 1; ++c) {
      R plane = 0;
#pragma unroll
      for (int b = -1; b <= 1; ++b) {
        const i64 q = pf + c * gf.sz + b * (i64)gf.Px;
        const R row = fma((R)0.5, cvt<R>(ldp<NC>(r + q)),
                          (R)0.25 * (cvt<R>(ldp<NC>(r + q - 1)) + cvt<R>(ldp<NC>(r + q + 1))));
        plane = fma(b == 0 ? (R)0.5 : (R)0.25, row, plane);
      }
      acc = fma(c == 0 ? (R)0.5 : (R)0.25, plane, acc);
    }
    bc[pc] = store_as<TV>(acc);
  }
};

// Trilinear prolongation and correction x += P e over the fine grid.  Along
// each axis a fine index i draws on coarse indices (i-1)>>1 and i>>1 with
// weight 1/2 each: for odd i both are the coincident coarse point (weight 1),
// for even i they are its two neighbours; index -1 and n_c are zero pads.
template <class R, class TV> struct OpProlong {
  Geom gc;
  const TV* e;
  TV* x;
  __device__ void prepare() {}
  template <bool NC> __device__ __forceinline__ void pt(const Geom&, int i, int j, int k, i64 p, double&,
                                                        double&) const {
    const int i0 = (i - 1) >> 1, i1 = i >> 1, j0 = (j - 1) >> 1, j1 = j >> 1, k0 = (k - 1) >> 1, k1 = k >> 1;
    const i64 a00 = gc.at(i0, j0, k0), a10 = gc.at(i0, j1, k0), a01 = gc.at(i0, j0, k1), a11 = gc.at(i0, j1, k1);
    const int di = i1 - i0;
    R s = cvt<R>(ldp<NC>(e + a00)) + cvt<R>(ldp<NC>(e + a00 + di));
    s += cvt<R>(ldp<NC>(e + a10)) + cvt<R>(ldp<NC>(e + a10 + di));
    s += cvt<R>(ldp<NC>(e + a01)) + cvt<R>(ldp<NC>(e + a01 + di));
    s += cvt<R>(ldp<NC>(e + a11)) + cvt<R>(ldp<NC>(e + a11 + di));
    x[p] = store_as<TV>(fma((R)0.125, s, cvt<R>(x[p])));
  }
};

// ---- outer CG (float64) ----------------------------------------------------
struct Scal {
  double bb, rr, rho, pq, rz_old, alpha, beta, rho_new, true_rr;
  int status;  // bit 0: non-finite, bit 1: breakdown (p.Ap <= 0)
  int pad;
};

// p = z + beta p in place (beta from the scalar block; z in the V-cycle's
// vector type).  beta = 0 on the first iteration, where p holds zeros.
template <class TZ> struct OpPUpd {
  const TZ* z;
  double* p;
  const Scal* sc;
  double beta;
  __device__ void prepare() { beta = sc->beta; }
  template <bool NC> __device__ __forceinline__ void pt(const Geom&, int, int, int, i64 i, double&, double&) const {
    p[i] = fma(beta, p[i], cvt<double>(ldp<NC>(z + i)));
  }
};

// q = A p with the stored float64 diagonal: q = D p - sum_q c_pq p_q;
// acc0 += p.q.  (8 float64 operations per point.)
struct OpApplyPQ {
  const double* p;
  double* q;
  const double* dg;
  const double *kx, *ky, *kz;
  __device__ void prepare() {}
  template <bool NC> __device__ __forceinline__ void pt(const Geom& g, int, int, int, i64 i, double& a0,
                                                        double&) const {
    double D;
    LdVec<NC, double, double> lp{p};
    const double S = stencil<NC, double>(g, i, lp, kx, ky, kz, D);
    const double pi = lp(i);
    const double qv = fma(ldp<NC>(dg + i), pi, -S);
    q[i] = qv;
    a0 = fma(pi, qv, a0);
  }
};

// x += alpha p, r -= alpha q; acc0 += r.r and, for the flexible (Polak-Ribiere)
// beta, acc1 += r_new . z_old (z still holds the previous preconditioned residual).
template <class TZ, bool FLEX> struct OpCgUpd {
  double* x;
  double* r;
  const double* p;
  const double* q;
  const TZ* z;
  const Scal* sc;
  double alpha;
  __device__ void prepare() { alpha = sc->alpha; }
  template <bool NC> __device__ __forceinline__ void pt(const Geom&, int, int, int, i64 i, double& a0,
                                                        double& a1) const {
    x[i] = fma(alpha, p[i], x[i]);
    const double rv = fma(-alpha, q[i], r[i]);
    r[i] = rv;
    a0 = fma(rv, rv, a0);
    if constexpr (FLEX) a1 = fma(rv, cvt<double>(ldp<NC>(z + i)), a1);
  }
};

// acc0 += a.b with b in the V-cycle's vector type
template <class TB> struct OpDot {
  const double* a;
  const TB* b;
  __device__ void prepare() {}
  template <bool NC> __device__ __forceinline__ void pt(const Geom&, int, int, int, i64 i, double& a0, double&) const {
    a0 = fma(ldp<NC>(a + i), cvt<double>(ldp<NC>(b + i)), a0);
  }
};

// ------------------------------------------------------------ reductions
// Deterministic block sum of (a0, a1): fixed xor-shuffle tree per warp, then
// warp 0 adds the per-warp sums in index order.  Thread 0 gets the result.
template <int NT>
__device__ __forceinline__ void block_sum2(double& a0, double& a1) {
  __shared__ double s0[NT / 32], s1[NT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
  }
  if (lane == 0) {
    s0[w] = a0;
    s1[w] = a1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0, t1 = 0;
    for (int q = 0; q < NT / 32; ++q) {
      t0 += s0[q];
      t1 += s1[q];
    }
    a0 = t0;
    a1 = t1;
  }
  __syncthreads();
}

}  // namespace mgdev
