// Galerkin coarse levels: A_{l+1} = R A_l P with R = P^T / 8 (the coarse
// operators of the paper's runs, Sec. 4.3 and Sec. 5).  With trilinear P the
// Galerkin operator of a 7-point (or 27-point) operator is a 27-point stencil
// with variable coefficients.
//
// Storage (padded level layout of mg_device.cuh): the operator is symmetric,
// so only the 13 couplings to the "forward" neighbours p + o (those with a
// positive linear offset) are stored, as w_o(p) = -(A)_{p,p+o}, in 13 arrays
// of the level's length (array o at w + o * wst).  The coupling to p - o is
// w_o(p - o), read from the neighbour.  Entries whose neighbour is not an
// interior point, and all pad slots, hold zero.  The diagonal is stored
// (dg) together with its inverse (dinv).
#pragma once
#include "mg_device.cuh"

namespace mgdev {

// Forward neighbour offsets (dx, dy, dz), those with dz*sz + dy*Px + dx > 0:
// o = 0: (1,0,0); o = 1..3: (o-2, 1, 0); o = 4..12: the nine (dx, dy) of the
// plane above, dx fastest.
__host__ __device__ __forceinline__ int g27_dx(int o) { return o == 0 ? 1 : o < 4 ? o - 2 : (o - 4) % 3 - 1; }
__host__ __device__ __forceinline__ int g27_dy(int o) { return o == 0 ? 0 : o < 4 ? 1 : (o - 4) / 3 - 1; }
__host__ __device__ __forceinline__ int g27_dz(int o) { return o < 4 ? 0 : 1; }

__host__ __device__ __forceinline__ int g27_off(const Geom& g, int o) {
  return g27_dz(o) * (int)g.sz + g27_dy(o) * g.Px + g27_dx(o);
}

// S_p = sum over the 26 neighbours q of w_pq u_q (forward and backward
// coupling of each stored offset in turn).
template <bool NC, class R, class TC, class U>
__device__ __forceinline__ R stencil27(const Geom& g, int p, const U& u, const TC* w, i64 wst) {
  R S = 0;
#pragma unroll
  for (int o = 0; o < 13; ++o) {
    const int off = g27_off(g, o);
    const TC* wo = w + (i64)o * wst;
    S = fma(cvt<R>(ldp<NC>(wo + p)), u(p + off), S);
    S = fma(cvt<R>(ldp<NC>(wo + p - off)), u(p - off), S);
  }
  return S;
}

// y = A u = D u - S
template <class R, class TV, class TC> struct OpApply27 {
  using Real = R;
  const TV* u;
  TV* y;
  const TC* w;
  i64 wst;
  const TV* dg;
  __device__ void prepare() {}
  template <bool NC> __device__ __forceinline__ void pt(const Geom& g, int, int, int, int p, double&, double&) const {
    LdVec<NC, R, TV> lu{u};
    const R S = stencil27<NC, R>(g, p, lu, w, wst);
    y[p] = store_as<TV>(cvt<R>(ldp<NC>(dg + p)) * lu(p) - S);
  }
};

// r = b - A x (acc0 += r.r)
template <class R, class TV, class TB, class TC> struct OpResidual27 {
  using Real = R;
  const TV* x;
  const TB* b;
  TV* r;
  const TC* w;
  i64 wst;
  const TV* dg;
  __device__ void prepare() {}
  template <bool NC> __device__ __forceinline__ void pt(const Geom& g, int, int, int, int p, double& acc,
                                                        double&) const {
    LdVec<NC, R, TV> lx{x};
    const R S = stencil27<NC, R>(g, p, lx, w, wst);
    const R rv = (cvt<R>(ldp<NC>(b + p)) + S) - cvt<R>(ldp<NC>(dg + p)) * lx(p);
    r[p] = store_as<TV>(rv);
    acc = fma((double)rv, (double)rv, acc);
  }
};

// Chebyshev steps 0 and 1 from a zero guess (as OpChebZero)
template <class R, class TV, class TC> struct OpChebZero27 {
  using Real = R;
  const TV* b;
  const TV* dinv;
  TV* xout;
  TV* dout;
  const TC* w;
  i64 wst;
  R c1, c2, inv_theta;
  __device__ void prepare() {}
  template <bool NC> __device__ __forceinline__ void pt(const Geom& g, int, int, int, int p, double&, double&) const {
    LdJac<NC, R, TV> lx{b, dinv, inv_theta};
    const R S = stencil27<NC, R>(g, p, lx, w, wst);
    const R x1 = lx(p);
    const R s = fma(cvt<R>(ldp<NC>(dinv + p)), cvt<R>(ldp<NC>(b + p)) + S, -x1);
    const R d1 = fma(c1, x1, c2 * s);
    xout[p] = store_as<TV>(x1 + d1);
    if (dout) dout[p] = store_as<TV>(d1);
  }
};

// Chebyshev step j (as OpChebStep) with the stored D^-1
template <class R, class TV, class TC> struct OpChebStep27 {
  using Real = R;
  const TV* x;
  const TV* dprev;
  const TV* b;
  const TV* dinv;
  TV* xout;
  TV* dout;
  const TC* w;
  i64 wst;
  R c1, c2, inv_theta;
  __device__ void prepare() {}
  template <bool NC> __device__ __forceinline__ void pt(const Geom& g, int, int, int, int p, double&, double&) const {
    LdVec<NC, R, TV> lx{x};
    const R S = stencil27<NC, R>(g, p, lx, w, wst);
    const R xp = lx(p);
    const R s = fma(cvt<R>(ldp<NC>(dinv + p)), cvt<R>(ldp<NC>(b + p)) + S, -xp);
    const R dn = dprev ? fma(c1, cvt<R>(ldp<NC>(dprev + p)), c2 * s) : s * inv_theta;
    xout[p] = store_as<TV>(xp + dn);
    if (dout) dout[p] = store_as<TV>(dn);
  }
};

// ------------------------------------------------------------ setup (float64)
// Fine operator of a Galerkin product: the 7-point operator of edge
// coefficients (kx, ky, kz; diagonal = their sum) or a stored 27-point one.
struct FineOp {
  Geom g;
  const double *kx, *ky, *kz;  // 7-point, or null
  const double *w, *dg;        // 27-point
  i64 wst;
};

// One coarse row of A_c = R A_f P per thread: the 27 fine rows i of R's
// stencil around the fine image of coarse point I, every stored entry a_ij
// of those rows, and the coarse interior nodes J that interpolate to fine
// node j (per axis: an odd fine index is a coarse node, weight 1; an even one
// lies between two, weight 1/2 each).  J - I is in {-1,0,1}^3.
__global__ void k_galerkin(FineOp F, Geom gc, double* w, double* dg) {
  const i64 n = gc.npts();
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x) {
    const int ci = (int)(t % gc.nx), cj = (int)((t / gc.nx) % gc.ny), ck = (int)(t / ((i64)gc.nx * gc.ny));
    double acc[27];
#pragma unroll
    for (int e = 0; e < 27; ++e) acc[e] = 0.0;
    const Geom& gf = F.g;
    for (int c = -1; c <= 1; ++c)
      for (int b = -1; b <= 1; ++b)
        for (int a = -1; a <= 1; ++a) {
          const int fi = 2 * ci + 1 + a, fj = 2 * cj + 1 + b, fk = 2 * ck + 1 + c;
          const double rI = (a ? 0.5 : 1.0) * (b ? 0.5 : 1.0) * (c ? 0.5 : 1.0) / 8.0;
          const int p = (int)gf.at(fi, fj, fk);
          // entries (dx, dy, dz, a_ij) of fine row i
          auto visit = [&](int dx, int dy, int dz, double aij) {
            const int gi = fi + dx, gj = fj + dy, gk = fk + dz;
            if (gi < 0 || gi >= gf.nx || gj < 0 || gj >= gf.ny || gk < 0 || gk >= gf.nz) return;
            int c0[3], c1[3];
            double w0[3], w1[3];
            const int gg[3] = {gi, gj, gk}, nc3[3] = {gc.nx, gc.ny, gc.nz};
            for (int ax = 0; ax < 3; ++ax) {
              if (gg[ax] & 1) {
                c0[ax] = c1[ax] = (gg[ax] - 1) / 2;
                w0[ax] = 1.0;
                w1[ax] = 0.0;
              } else {
                c0[ax] = gg[ax] / 2 - 1;
                c1[ax] = gg[ax] / 2;
                w0[ax] = w1[ax] = 0.5;
              }
            }
            for (int sz_ = 0; sz_ < 2; ++sz_)
              for (int sy = 0; sy < 2; ++sy)
                for (int sx = 0; sx < 2; ++sx) {
                  const double px = sx ? w1[0] : w0[0], py = sy ? w1[1] : w0[1], pz = sz_ ? w1[2] : w0[2];
                  if (px == 0.0 || py == 0.0 || pz == 0.0) continue;
                  const int Jx = sx ? c1[0] : c0[0], Jy = sy ? c1[1] : c0[1], Jz = sz_ ? c1[2] : c0[2];
                  if (Jx < 0 || Jx >= nc3[0] || Jy < 0 || Jy >= nc3[1] || Jz < 0 || Jz >= nc3[2]) continue;
                  acc[((Jz - ck + 1) * 3 + (Jy - cj + 1)) * 3 + (Jx - ci + 1)] += rI * aij * (px * py * pz);
                }
          };
          if (F.kx) {
            const int sy = gf.Px, sz = (int)gf.sz;
            const double cxm = F.kx[p - 1], cxp = F.kx[p], cym = F.ky[p - sy], cyp = F.ky[p], czm = F.kz[p - sz],
                         czp = F.kz[p];
            visit(0, 0, -1, -czm);
            visit(0, -1, 0, -cym);
            visit(-1, 0, 0, -cxm);
            visit(0, 0, 0, ((cxm + cxp) + (cym + cyp)) + (czm + czp));
            visit(1, 0, 0, -cxp);
            visit(0, 1, 0, -cyp);
            visit(0, 0, 1, -czp);
          } else {
            visit(0, 0, 0, F.dg[p]);
            for (int o = 0; o < 13; ++o) {
              const int off = g27_off(gf, o);
              visit(g27_dx(o), g27_dy(o), g27_dz(o), -F.w[(i64)o * F.wst + p]);
              visit(-g27_dx(o), -g27_dy(o), -g27_dz(o), -F.w[(i64)o * F.wst + p - off]);
            }
          }
        }
    const i64 P = gc.at(ci, cj, ck);
    dg[P] = acc[13];
    for (int o = 0; o < 13; ++o) {
      const int X = ci + g27_dx(o), Y = cj + g27_dy(o), Z = ck + g27_dz(o);
      if (X < 0 || X >= gc.nx || Y < 0 || Y >= gc.ny || Z < 0 || Z >= gc.nz) continue;
      w[(i64)o * gc.len + P] = -acc[((g27_dz(o) + 1) * 3 + (g27_dy(o) + 1)) * 3 + (g27_dx(o) + 1)];
    }
  }
}

// Gershgorin bound of D^-1 A: max over rows of sum_j |a_ij| / a_ii, as the
// bits of a positive double (integer order = value order) in *out.
__global__ void k_gershgorin27(const double* w, const double* dg, Geom g, unsigned long long* out) {
  const i64 n = g.npts();
  double best = 0.0;
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.nx), j = (int)((t / g.nx) % g.ny), k = (int)(t / ((i64)g.nx * g.ny));
    const int p = (int)g.at(i, j, k);
    double s = fabs(dg[p]);
    for (int o = 0; o < 13; ++o) {
      const int off = g27_off(g, o);
      s += fabs(w[(i64)o * g.len + p]) + fabs(w[(i64)o * g.len + p - off]);
    }
    const double v = s / dg[p];
    best = v > best ? v : best;
  }
  atomicMax(out, (unsigned long long)__double_as_longlong(best));
}

// D^-1 (and D) of a 27-point level in the V-cycle precision
template <class TV> __global__ void k_diag27(const double* dg64, TV* dg, TV* dinv, Geom g) {
  const i64 n = g.npts();
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.nx), j = (int)((t / g.nx) % g.ny), k = (int)(t / ((i64)g.nx * g.ny));
    const i64 p = g.at(i, j, k);
    dg[p] = store_as<TV>(dg64[p]);
    dinv[p] = store_as<TV>(1.0 / dg64[p]);
  }
}

// Dense n x n matrix of a 27-point level (interior numbering (k*ny + j)*nx + i)
__global__ void k_assemble_dense27(const double* w, const double* dg, Geom g, double* A) {
  const i64 n = g.npts();
  for (i64 u = blockIdx.x * (i64)blockDim.x + threadIdx.x; u < n; u += (i64)gridDim.x * blockDim.x) {
    const int i = (int)(u % g.nx), j = (int)((u / g.nx) % g.ny), k = (int)(u / ((i64)g.nx * g.ny));
    const i64 p = g.at(i, j, k);
    A[u * n + u] = dg[p];
    for (int o = 0; o < 13; ++o) {
      const int X = i + g27_dx(o), Y = j + g27_dy(o), Z = k + g27_dz(o);
      if (X < 0 || X >= g.nx || Y < 0 || Y >= g.ny || Z < 0 || Z >= g.nz) continue;
      const i64 v = ((i64)Z * g.ny + Y) * g.nx + X;
      const double a = -w[(i64)o * g.len + p];
      A[u * n + v] = a;
      A[v * n + u] = a;
    }
  }
}

}  // namespace mgdev
