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
#include <string.h>

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
// float <-> double conversions on the integer pipe.  On GB300 the float64 pipe
// (which also executes F2F conversions) is the scarce unit of the outer CG, so
// the float32 vectors that meet float64 ones there are converted with bit
// operations instead:
//   f2d_bits: exact for zeros, normal numbers, infinities and NaNs; a
//             subnormal float becomes a signed zero;
//   d2f_bits: round to nearest, ties to even, exactly as a float64 -> float32
//             conversion for every result in the normal float range; results
//             below it become a signed zero, above it infinity.
__host__ __device__ __forceinline__ unsigned long long dbits(double d) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(d);
#else
  unsigned long long u;
  memcpy(&u, &d, 8);
  return u;
#endif
}
__host__ __device__ __forceinline__ double bitsd(unsigned long long u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double d;
  memcpy(&d, &u, 8);
  return d;
#endif
}
__host__ __device__ __forceinline__ unsigned fbits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  unsigned u;
  memcpy(&u, &f, 4);
  return u;
#endif
}
__host__ __device__ __forceinline__ float bitsf(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}
__host__ __device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = fbits(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long mant = e == 0 ? 0ull : (unsigned long long)(u & 0x7fffffu) << 29;
  const unsigned long long E = e == 0 ? 0ull : (e == 255 ? 2047ull : (unsigned long long)(e + 896u));
  return bitsd(sign | (E << 52) | mant);
}
__host__ __device__ __forceinline__ float d2f_bits(double d) {
  const unsigned long long u = dbits(d);
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7ff);
  const unsigned long long m = u & 0xfffffffffffffull;
  if (e == 0x7ff) return bitsf(sign | 0x7f800000u | (m ? 0x400000u : 0u));  // infinity, NaN
  const int fe = e - 1023 + 127;
  if (fe >= 255) return bitsf(sign | 0x7f800000u);
  if (fe <= 0) return bitsf(sign);
  unsigned keep = (unsigned)(m >> 29);
  const unsigned long long rem = m & 0x1fffffffull;
  if (rem > 0x10000000ull || (rem == 0x10000000ull && (keep & 1u))) ++keep;
  const unsigned bits = ((unsigned)fe << 23) + keep;  // a mantissa carry moves into the exponent
  if ((bits >> 23) >= 255u) return bitsf(sign | 0x7f800000u);
  return bitsf(sign | bits);
}

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
// NC = false is a plain coherent load (the bottom kernel reads what its own
// threads, or its cluster's, wrote before a barrier).
template <bool NC, class T> __device__ __forceinline__ T ldp(const T* p) {
  if constexpr (NC) return __ldg(p);
  else return *p;
}

// Programmatic dependent launch: a kernel launched while the previous one in
// the stream is still finishing waits here before touching global memory
// (a no-op for ordinary launches), and lets the next kernel launch once its
// own main loop is done.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ------------------------------------------------------------ loaders
template <bool NC, class R, class T> struct LdVec {
  const T* a;
  __device__ __forceinline__ R operator()(int q) const { return cvt<R>(ldp<NC>(a + q)); }
};
// First Chebyshev iterate from a zero guess: x_1 = D^-1 b / theta.
template <bool NC, class R, class TV> struct LdJac {
  const TV* b;
  const TV* dinv;
  R inv_theta;
  __device__ __forceinline__ R operator()(int q) const {
    return inv_theta * (cvt<R>(ldp<NC>(dinv + q)) * cvt<R>(ldp<NC>(b + q)));
  }
};
// S_p = sum_q c_pq u_q and D_p = sum_q c_pq at interior point p.
template <bool NC, class R, class TC, class U>
__device__ __forceinline__ R stencil(const Geom& g, int p, const U& u, const TC* kx, const TC* ky, const TC* kz,
                                     R& D) {
  const int sy = g.Px, sz = (int)g.sz;
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

// D^-1 at a point: in float32 it is recomputed from the six coefficients the
// stencil already loaded (the same sum and division that produced the stored
// inverse, so the value is identical and 4 bytes per point are not read); in
// float64, where the float64 pipe is the bottleneck, the stored inverse is read.
template <bool NC, class R, class TV>
__device__ __forceinline__ R inv_diag(R D, const TV* dinv_p) {
  if constexpr (sizeof(R) == 4) return (R)1 / D;
  else return cvt<R>(ldp<NC>(dinv_p));
}

// ------------------------------------------------------------ point operations
// Every op exposes  template<bool NC> void pt(g, i, j, k, p, acc0, acc1)
// and  prepare()  (called once per thread before the point loop).

// y = A u
template <class R, class TV, class TC> struct OpApply {
  using Real = R;
  const TV* u;
  TV* y;
  const TC *kx, *ky, *kz;
  __device__ void prepare() {}
  template <bool NC> __device__ __forceinline__ void pt(const Geom& g, int, int, int, int p, double&, double&) const {
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
  using Real = R;
  const TV* x;
  const TV* dprev;  // null for j = 0
  const TV* b;
  const TV* dinv;
  TV* xout;
  TV* dout;  // null when d_j is not needed afterwards
  const TC *kx, *ky, *kz;
  R c1, c2, inv_theta;
  __device__ void prepare() {}
  // performs the step at p and returns x_{j+1}
  template <bool NC> __device__ __forceinline__ R step(const Geom& g, int p) const {
    R D;
    LdVec<NC, R, TV> lx{x};
    R S = stencil<NC, R>(g, p, lx, kx, ky, kz, D);
    const R xp = lx(p);
    const R s = fma(inv_diag<NC>(D, dinv + p), cvt<R>(ldp<NC>(b + p)) + S, -xp);
    const R dn = dprev ? fma(c1, cvt<R>(ldp<NC>(dprev + p)), c2 * s) : s * inv_theta;
    const R xn = xp + dn;
    xout[p] = store_as<TV>(xn);
    if (dout) dout[p] = store_as<TV>(dn);
    return xn;
  }
  template <bool NC> __device__ __forceinline__ void pt(const Geom& g, int, int, int, int p, double&, double&) const {
    step<NC>(g, p);
  }
};

// Steps 0 and 1 of a sweep from a zero initial guess in one pass:
//   x_1 = d_0 = D^-1 b / theta (formed on the fly at the 7 stencil points),
//   s_1 = D^-1 (b - A x_1), d_1 = c1 d_0 + c2 s_1, x_2 = x_1 + d_1.
template <class R, class TV, class TC> struct OpChebZero {
  using Real = R;
  const TV* b;
  const TV* dinv;
  TV* xout;
  TV* dout;
  const TC *kx, *ky, *kz;
  R c1, c2, inv_theta;
  __device__ void prepare() {}
  template <bool NC> __device__ __forceinline__ void pt(const Geom& g, int, int, int, int p, double&, double&) const {
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
  using Real = R;
  const TV* b;
  const TV* dinv;
  TV* xout;
  R inv_theta;
  __device__ void prepare() {}
  template <bool NC> __device__ __forceinline__ void pt(const Geom&, int, int, int, int p, double&, double&) const {
    xout[p] = store_as<TV>(inv_theta * (cvt<R>(ldp<NC>(dinv + p)) * cvt<R>(ldp<NC>(b + p))));
  }
};

// Chebyshev step 0 from a zero guess stored as both iterate and direction,
// x = d = D^-1 b / theta (the value LdJac forms), so that step 1 runs as an
// ordinary step.  The float64 forms use it: forming D^-1 b / theta again at
// every neighbour of every point, as the fused zero-guess step does, costs
// two float64 multiplications per neighbour on GB300's slow float64 pipe.
// Step 1 from the stored values gives the fused step's result bit for bit.
template <class R, class TV> struct OpChebStart {
  using Real = R;
  const TV* b;
  const TV* dinv;
  TV* x;
  TV* d;
  R inv_theta;
  __device__ void prepare() {}
  template <bool NC> __device__ __forceinline__ void pt(const Geom&, int, int, int, int p, double&, double&) const {
    const TV v = store_as<TV>(inv_theta * (cvt<R>(ldp<NC>(dinv + p)) * cvt<R>(ldp<NC>(b + p))));
    x[p] = v;
    d[p] = v;
  }
};

// r = b - A x
template <class R, class TV, class TB, class TC> struct OpResidual {
  using Real = R;
  const TV* x;
  const TB* b;
  TV* r;
  const TC *kx, *ky, *kz;
  __device__ void prepare() {}
  template <bool NC> __device__ __forceinline__ void pt(const Geom& g, int, int, int, int p, double& acc,
                                                        double&) const {
    R D;
    LdVec<NC, R, TV> lx{x};
    R S = stencil<NC, R>(g, p, lx, kx, ky, kz, D);
    const R rv = (cvt<R>(ldp<NC>(b + p)) + S) - D * lx(p);
    r[p] = store_as<TV>(rv);
    acc = fma((double)rv, (double)rv, acc);
  }
};

// r = b - A x in float64 with the stored diagonal dg (the finest level's sum
// of the six edge coefficients, in stencil()'s order, so the value is that of
// OpResidual bit for bit).  On GB300's float64 pipe, forming D again would cost
// five additions per point in a kernel that the pipe bounds.
template <class TB> struct OpResidualD {
  using Real = double;
  const double* x;
  const TB* b;
  double* r;
  const double* dg;
  const double *kx, *ky, *kz;
  __device__ void prepare() {}
  template <bool NC> __device__ __forceinline__ void pt(const Geom& g, int, int, int, int p, double& acc,
                                                        double&) const {
    double D;
    LdVec<NC, double, double> lx{x};
    const double S = stencil<NC, double>(g, p, lx, kx, ky, kz, D);
    const double rv = (cvt<double>(ldp<NC>(b + p)) + S) - ldp<NC>(dg + p) * lx(p);
    r[p] = rv;
    acc = fma(rv, rv, acc);
  }
};

// Full weighting bc = R r, R = P^T / 8: weights (1/4, 1/2, 1/4) per axis
// around fine point (2i+1, 2j+1, 2k+1), the image of coarse point (i,j,k).
// Runs over the coarse grid; gf is the fine geometry.
template <class R, class TV> struct OpRestrict {
  using Real = R;
  Geom gf;
  const TV* r;
  TV* bc;
  __device__ void prepare() {}
  template <bool NC> __device__ __forceinline__ void pt(const Geom&, int i, int j, int k, int pc, double&,
                                                        double&) const {
    const int pf = (int)gf.at(2 * i + 1, 2 * j + 1, 2 * k + 1);
    R acc = 0;
#pragma unroll
    for (int c = -1; c <= 1; ++c) {
      R plane = 0;
#pragma unroll
      for (int b = -1; b <= 1; ++b) {
        const int q = pf + c * (int)gf.sz + b * gf.Px;
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
// The eight terms are summed per coarse column first (the two rows and two
// planes of column i0, then of column i1), so that the vector kernel, which
// updates several fine points of a row, forms each column's sum once and
// shares it: x += (Y(i0) + Y(i1)) / 8 with Y(c) = (e(c,j0,k0) + e(c,j0,k1)) +
// (e(c,j1,k0) + e(c,j1,k1)).  (Half the floating-point additions of a sum
// taken point by point, which matters in float64 on GB300.)
template <class R, class TV> struct OpProlong {
  using Real = R;
  Geom gc;
  const TV* e;
  TV* x;
  __device__ void prepare() {}
  template <bool NC> __device__ __forceinline__ void pt(const Geom&, int i, int j, int k, int p, double&,
                                                        double&) const {
    const int i0 = (i - 1) >> 1, i1 = i >> 1, j0 = (j - 1) >> 1, j1 = j >> 1, k0 = (k - 1) >> 1, k1 = k >> 1;
    const int a00 = (int)gc.at(i0, j0, k0), a10 = (int)gc.at(i0, j1, k0), a01 = (int)gc.at(i0, j0, k1),
              a11 = (int)gc.at(i0, j1, k1);
    const int di = i1 - i0;
    auto col = [&](int o) {
      return (cvt<R>(ldp<NC>(e + a00 + o)) + cvt<R>(ldp<NC>(e + a01 + o))) +
             (cvt<R>(ldp<NC>(e + a10 + o)) + cvt<R>(ldp<NC>(e + a11 + o)));
    };
    const R s = col(0) + col(di);
    x[p] = store_as<TV>(fma((R)0.125, s, cvt<R>(x[p])));
  }
};

// ---- outer CG (float64) ----------------------------------------------------
struct Scal {
  double bb, rr, rho, pq, rz_old, alpha, beta, rho_new, true_rr;
  int status;  // bit 0: non-finite, bit 1: breakdown (p.Ap <= 0)
  int pad;
};

// q = A p with the stored float64 diagonal: q = D p - sum_q c_pq p_q;
// acc0 += p.q.  (8 float64 operations per point.)
struct OpApplyPQ {
  using Real = float;  // no spills at 40 registers; float64-pipe bound either way
  const double* p;
  double* q;
  const double* dg;
  const double *kx, *ky, *kz;
  __device__ void prepare() {}
  template <bool NC> __device__ __forceinline__ void pt(const Geom& g, int, int, int, int i, double& a0,
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

__device__ __forceinline__ double to_double(float v) { return f2d_bits(v); }
__device__ __forceinline__ double to_double(double v) { return v; }

// ---- linear (pointwise) kernels over whole padded arrays ---------------------
// Pad slots hold zeros in every vector and stay zero under these updates, so
// the pointwise CG kernels run over [0, len) with 4 consecutive elements per
// thread and 16-byte vector accesses (len is a multiple of 8).
__device__ __forceinline__ void ld4(const double* p, double v[4]) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p + 2));
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void ld4(const float* p, double v[4]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = f2d_bits(a.x); v[1] = f2d_bits(a.y); v[2] = f2d_bits(a.z); v[3] = f2d_bits(a.w);
}
__device__ __forceinline__ void st4(double* p, const double v[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void st4(float* p, const double v[4]) {
  reinterpret_cast<float4*>(p)[0] = make_float4(d2f_bits(v[0]), d2f_bits(v[1]), d2f_bits(v[2]), d2f_bits(v[3]));
}

// x += alpha p (the update of the previous iteration, deferred to this pass,
// which reads p anyway), then p = z + beta p.  alpha = 0 on the first iteration.
template <class TZ> struct LinPUpd {
  const TZ* z;
  double* p;
  double* x;
  const Scal* sc;
  double alpha, beta;
  __device__ void prepare() {
    alpha = sc->alpha;
    beta = sc->beta;
  }
  __device__ __forceinline__ void pt4(i64 t, double&, double&) const {
    double zv[4], pv[4], xv[4];
    ld4(z + t, zv);
    ld4(p + t, pv);
    ld4(x + t, xv);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      xv[u] = fma(alpha, pv[u], xv[u]);
      pv[u] = fma(beta, pv[u], zv[u]);
    }
    st4(x + t, xv);
    st4(p + t, pv);
  }
};

// x += alpha p (the last iteration's update at exit)
struct LinXUpd {
  double* x;
  const double* p;
  const Scal* sc;
  double alpha;
  __device__ void prepare() { alpha = sc->alpha; }
  __device__ __forceinline__ void pt4(i64 t, double&, double&) const {
    double xv[4], pv[4];
    ld4(x + t, xv);
    ld4(p + t, pv);
#pragma unroll
    for (int u = 0; u < 4; ++u) xv[u] = fma(alpha, pv[u], xv[u]);
    st4(x + t, xv);
  }
};

// r -= alpha q, acc0 += r.r, acc1 += r.z_old (FLEX); with B32 also
// b32 = (float) r, the float32 right-hand side of the next V-cycle.
template <class TZ, bool FLEX, bool B32> struct LinCgUpd {
  double* r;
  const double* q;
  const TZ* z;
  float* b32;
  const Scal* sc;
  double alpha;
  __device__ void prepare() { alpha = sc->alpha; }
  __device__ __forceinline__ void pt4(i64 t, double& a0, double& a1) const {
    double rv[4], qv[4];
    ld4(r + t, rv);
    ld4(q + t, qv);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      rv[u] = fma(-alpha, qv[u], rv[u]);
      a0 = fma(rv[u], rv[u], a0);
    }
    if constexpr (FLEX) {
      double zv[4];
      ld4(z + t, zv);
#pragma unroll
      for (int u = 0; u < 4; ++u) a1 = fma(rv[u], zv[u], a1);
    }
    st4(r + t, rv);
    if constexpr (B32) st4(b32 + t, rv);
  }
};

// acc0 += a.b for two vectors of the same (V-cycle) precision
template <class TA> struct LinDotT {
  const TA* a;
  const TA* b;
  __device__ void prepare() {}
  __device__ __forceinline__ void pt4(i64 t, double& a0, double&) const {
    double av[4], bv[4];
    ld4(a + t, av);
    ld4(b + t, bv);
#pragma unroll
    for (int u = 0; u < 4; ++u) a0 = fma(av[u], bv[u], a0);
  }
};

// acc0 += a.b
template <class TB> struct LinDot {
  const double* a;
  const TB* b;
  __device__ void prepare() {}
  __device__ __forceinline__ void pt4(i64 t, double& a0, double&) const {
    double av[4], bv[4];
    ld4(a + t, av);
    ld4(b + t, bv);
#pragma unroll
    for (int u = 0; u < 4; ++u) a0 = fma(av[u], bv[u], a0);
  }
};

// Final post-smoothing step on the finest level with the CG dot product rho
// fused in, accumulated in float64: rho = b.z with z = x_{j+1} the V-cycle's
// output as stored and b its finest right-hand side as the V-cycle read it.
// In the float64 form b is the outer residual r itself, so rho = r.z.  In the
// mixed forms b is the float32 rounding of r, and rho = b^T M b is the
// quadratic form of the preconditioner M that the float32 V-cycle applies
// (z = M b); it differs from r.z by at most one float32 rounding of each r
// entry and saves the pass's float64 read of r.
template <class R, class TV, class TC> struct OpChebStepDot {
  using Real = R;
  OpChebStep<R, TV, TC> step;
  __device__ void prepare() {}
  template <bool NC> __device__ __forceinline__ void pt(const Geom& g, int, int, int, int p, double& a0,
                                                        double&) const {
    const R xn = step.template step<NC>(g, p);
    a0 = fma(to_double(ldp<NC>(step.b + p)), to_double(store_as<TV>(xn)), a0);
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
