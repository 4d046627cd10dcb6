// Kernels of the multigrid-preconditioned CG solve (see mg_device.cuh for the
// data layout and the per-point operations).
#pragma once
#include "mg_device.cuh"
#include "mg_g27.cuh"

namespace mgdev {

constexpr int ZM_THREADS = 128;  // z-marching tile: 32 (x) by 4 (y) columns
constexpr int ZM_TX = 32, ZM_TY = 4;
// Resident blocks per SM requested from the compiler: 8 blocks of 128 threads
// (64 registers per thread).  Measured on the finest smoother step at 257^3:
// 32x4 tiles with 8 resident blocks and short plane chunks beat 32x8 tiles by
// ~30% (the larger blocks leave a partial last wave).
template <class Op> struct ZmMinBlocks { static constexpr int value = 8; };

// Multi-block z-marching driver: each thread owns one (i, j) column of a
// 32 x 8 tile and walks planes [k0, k1).  With RED the per-thread sums are
// reduced per block and written to partials[blockLinear] (and
// partials[stride + blockLinear] for the second sum).
template <class Op, bool RED>
__global__ void __launch_bounds__(ZM_THREADS, ZmMinBlocks<Op>::value) k_zmarch(Op op, Geom g, int kchunk, double* partials, int stride) {
  pdl_wait();
  op.prepare();
  const int i = blockIdx.x * ZM_TX + (threadIdx.x & 31);
  const int j = blockIdx.y * ZM_TY + (threadIdx.x >> 5);  // ZM_TX == 32
  const int k0 = blockIdx.z * kchunk;
  const int k1 = min(k0 + kchunk, g.nz);
  double a0 = 0.0, a1 = 0.0;
  if (i < g.nx && j < g.ny) {
    int p = (int)g.at(i, j, k0);
    const int sz = (int)g.sz;
    for (int k = k0; k < k1; ++k, p += sz) op.template pt<true>(g, i, j, k, p, a0, a1);
  }
  pdl_trigger();
  if constexpr (RED) {
    block_sum2<ZM_THREADS>(a0, a1);
    if (threadIdx.x == 0) {
      const int b = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      partials[b] = a0;
      partials[stride + b] = a1;
    }
  }
}

// Linear driver over whole padded arrays: 4 consecutive elements per thread
// per step, fixed grid, deterministic per-block sums as in k_zmarch.
constexpr int LIN_THREADS = 256;
template <class Op, bool RED>
__global__ void __launch_bounds__(LIN_THREADS) k_linear(Op op, i64 lo, i64 n, double* partials, int stride) {
  pdl_wait();
  op.prepare();
  double a0 = 0.0, a1 = 0.0;
  const i64 step = (i64)gridDim.x * LIN_THREADS * 4;
  for (i64 t = lo + ((i64)blockIdx.x * LIN_THREADS + threadIdx.x) * 4; t < n; t += step) op.pt4(t, a0, a1);
  pdl_trigger();
  if constexpr (RED) {
    block_sum2<LIN_THREADS>(a0, a1);
    if (threadIdx.x == 0) {
      partials[blockIdx.x] = a0;
      partials[stride + blockIdx.x] = a1;
    }
  }
}

// The bottom kernel runs as one thread block (CL = false) or as one
// thread-block cluster (CL = true): the blocks of the cluster split every
// pass, and a cluster barrier with release / acquire semantics separates the
// passes.
template <bool CL> struct BotSync {
  static __device__ __forceinline__ unsigned rank() {
    unsigned r = 0;
    if constexpr (CL) asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
  }
  static __device__ __forceinline__ unsigned blocks() {
    unsigned n = 1;
    if constexpr (CL) asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(n));
    return n;
  }
  static __device__ __forceinline__ void sync() {
    if constexpr (CL)
      asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    else __syncthreads();
  }
};

// Loop of the bottom kernel's threads (of one block, or of all blocks of the
// cluster) over all interior points of g.  The iteration space is padded to
// powers of two in x and y so the point indices come from shifts and masks
// instead of divisions.
template <bool CL = false, class Op>
__device__ __forceinline__ void block_for(const Op& op, const Geom& g) {
  const int lx = 32 - __clz(g.nx - 1), ly = 32 - __clz(g.ny - 1);  // ceil(log2)
  const unsigned n = (unsigned)g.nz << (lx + ly);
  const unsigned mx = (1u << lx) - 1, my = (1u << ly) - 1;
  double a0 = 0, a1 = 0;
  const unsigned t0 = BotSync<CL>::rank() * blockDim.x + threadIdx.x, step = BotSync<CL>::blocks() * blockDim.x;
  for (unsigned t = t0; t < n; t += step) {
    const int i = (int)(t & mx), j = (int)((t >> lx) & my), k = (int)(t >> (lx + ly));
    if (i < g.nx && j < g.ny) op.template pt<false>(g, i, j, k, (int)g.at(i, j, k), a0, a1);
  }
}

// ------------------------------------------------------------ layout conversion
// dense full-grid float64 (Nz,Ny,Nx) -> padded interior array of type T
template <class T>
__global__ void k_pack(const double* __restrict__ src, T* __restrict__ dst, Geom g) {
  const i64 n = g.npts();
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.nx);
    const i64 r = t / g.nx;
    const int j = (int)(r % g.ny);
    const int k = (int)(r / g.ny);
    const int Nx = g.nx + 2, Ny = g.ny + 2;
    dst[g.at(i, j, k)] = store_as<T>(src[((i64)(k + 1) * Ny + (j + 1)) * Nx + (i + 1)]);
  }
}

// padded interior array of type T -> dense full-grid float64 with zero
// boundary, full-grid planes K = kfirst .. klast (0 .. nz+1 for the whole
// grid; a z-slab writes only the planes it owns)
template <class T>
__global__ void k_unpack(const T* __restrict__ src, double* __restrict__ dst, Geom g, int kfirst, int klast) {
  const int Nx = g.nx + 2, Ny = g.ny + 2;
  const i64 n = (i64)Nx * Ny * (klast - kfirst + 1);
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x) {
    const int I = (int)(t % Nx);
    const i64 r = t / Nx;
    const int J = (int)(r % Ny);
    const int K = kfirst + (int)(r / Ny);
    const bool in = I >= 1 && I <= g.nx && J >= 1 && J <= g.ny && K >= 1 && K <= g.nz;
    dst[((i64)K * Ny + J) * Nx + I] = in ? cvt<double>(src[g.at(I - 1, J - 1, K - 1)]) : 0.0;
  }
}

// elementwise conversion of whole padded arrays (pads stay zero)
template <class TD, class TS>
__global__ void k_cast(const TS* __restrict__ src, TD* __restrict__ dst, i64 n) {
  pdl_wait();
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x)
    dst[t] = store_as<TD>(cvt<double>(src[t]));
}

// ------------------------------------------------------------ setup
// k (or ln k) per cell -> k, with a flag for non-positive / non-finite values.
__global__ void k_cells_init(double* kc, i64 n, int is_log, int* bad) {
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x) {
    double v = kc[t];
    if (is_log) v = exp(v);
    if (!(v > 0.0) || !isfinite(v)) atomicOr(bad, 1);
    kc[t] = v;
  }
}

// Coarse cell k as a mean of its 8 children: 0 arithmetic, 1 geometric, 2 harmonic.
__global__ void k_coarsen_cells(const double* __restrict__ kf, double* __restrict__ kc, int cx, int cy, int cz,
                                int rule) {
  const i64 n = (i64)cx * cy * cz;
  const int fx = 2 * cx, fy = 2 * cy;
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x) {
    const int ci = (int)(t % cx);
    const i64 r = t / cx;
    const int cj = (int)(r % cy);
    const int ck = (int)(r / cy);
    double s = 0.0;
    for (int c = 0; c < 2; ++c)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
          const double v = kf[((i64)(2 * ck + c) * fy + (2 * cj + b)) * fx + (2 * ci + a)];
          s += rule == 0 ? v : rule == 1 ? log(v) : 1.0 / v;
        }
    kc[t] = rule == 0 ? s * 0.125 : rule == 1 ? exp(s * 0.125) : 8.0 / s;
  }
}

// Mean of the 4 cells sharing an edge: harmonic (face_rule 0) or arithmetic.
__device__ __forceinline__ double edge_mean(double a, double b, double c, double d, int face_rule) {
  return face_rule ? 0.25 * ((a + b) + (c + d)) : 4.0 / ((1.0 / a + 1.0 / b) + (1.0 / c + 1.0 / d));
}

// Edge coefficients h_a^-2 k_e into the padded layout.  Thread (i,j,k) over
// [-1,nx) x [-1,ny) x [-1,nz) writes the +x edge of point (i,j,k) when j,k are
// interior, the +y edge when i,k are, the +z edge when i,j are.  Cells are the
// dense (nz+1)(ny+1)(nx+1) array of this level.
template <class TC>
__global__ void k_build_coef(const double* __restrict__ kc, Geom g, double ihx2, double ihy2, double ihz2,
                             int face_rule, TC* kx, TC* ky, TC* kz, double* kx64, double* ky64, double* kz64) {
  const int bx = g.nx + 1, by = g.ny + 1, bz = g.nz + 1;
  const i64 n = (i64)bx * by * bz;
  const int cx = g.nx + 1, cy = g.ny + 1;  // cells per axis
  auto cell = [&](int ci, int cj, int ck) { return kc[((i64)ck * cy + cj) * cx + ci]; };
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x) {
    const int i = (int)(t % bx) - 1;
    const i64 r = t / bx;
    const int j = (int)(r % by) - 1;
    const int k = (int)(r / by) - 1;
    const i64 p = g.at(i, j, k);
    if (j >= 0 && k >= 0) {  // edge (i,j,k)-(i+1,j,k): cells (i+1, j..j+1, k..k+1)
      const double v = ihx2 * edge_mean(cell(i + 1, j, k), cell(i + 1, j + 1, k), cell(i + 1, j, k + 1),
                                        cell(i + 1, j + 1, k + 1), face_rule);
      if (kx) kx[p] = store_as<TC>(v);
      if (kx64) kx64[p] = v;
    }
    if (i >= 0 && k >= 0) {  // edge (i,j,k)-(i,j+1,k): cells (i..i+1, j+1, k..k+1)
      const double v = ihy2 * edge_mean(cell(i, j + 1, k), cell(i + 1, j + 1, k), cell(i, j + 1, k + 1),
                                        cell(i + 1, j + 1, k + 1), face_rule);
      if (ky) ky[p] = store_as<TC>(v);
      if (ky64) ky64[p] = v;
    }
    if (i >= 0 && j >= 0) {  // edge (i,j,k)-(i,j,k+1): cells (i..i+1, j..j+1, k+1)
      const double v = ihz2 * edge_mean(cell(i, j, k + 1), cell(i + 1, j, k + 1), cell(i, j + 1, k + 1),
                                        cell(i + 1, j + 1, k + 1), face_rule);
      if (kz) kz[p] = store_as<TC>(v);
      if (kz64) kz64[p] = v;
    }
  }
}

// float64 diagonal D = sum of the 6 float64 edge coefficients (outer operator)
__global__ void k_diag64(const double* kx, const double* ky, const double* kz, double* dg, Geom g) {
  const i64 n = g.npts();
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.nx);
    const i64 r = t / g.nx;
    const int j = (int)(r % g.ny);
    const int k = (int)(r / g.ny);
    const i64 p = g.at(i, j, k);
    dg[p] = ((kx[p - 1] + kx[p]) + (ky[p - g.Px] + ky[p])) + (kz[p - g.sz] + kz[p]);
  }
}

// dinv = 1 / sum of the 6 stored edge coefficients (summed in precision R)
template <class R, class TV, class TC>
__global__ void k_dinv(const TC* kx, const TC* ky, const TC* kz, TV* dinv, Geom g) {
  const i64 n = g.npts();
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.nx);
    const i64 r = t / g.nx;
    const int j = (int)(r % g.ny);
    const int k = (int)(r / g.ny);
    const i64 p = g.at(i, j, k);
    const R D = ((cvt<R>(kx[p - 1]) + cvt<R>(kx[p])) + (cvt<R>(ky[p - g.Px]) + cvt<R>(ky[p]))) +
                (cvt<R>(kz[p - g.sz]) + cvt<R>(kz[p]));
    dinv[p] = store_as<TV>((R)1 / D);
  }
}

// Dense float64 operator of a (small) level in compact interior numbering.
__global__ void k_assemble_dense(const double* kx, const double* ky, const double* kz, Geom g, double* A) {
  const int n = (int)g.npts();
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
    const int i = u % g.nx, j = (u / g.nx) % g.ny, k = u / (g.nx * g.ny);
    const i64 p = g.at(i, j, k);
    double* row = A + (i64)u * n;
    for (int v = 0; v < n; ++v) row[v] = 0.0;
    const double c[6] = {kx[p - 1], kx[p], ky[p - g.Px], ky[p], kz[p - g.sz], kz[p]};
    row[u] = ((c[0] + c[1]) + (c[2] + c[3])) + (c[4] + c[5]);
    if (i > 0) row[u - 1] = -c[0];
    if (i < g.nx - 1) row[u + 1] = -c[1];
    if (j > 0) row[u - g.nx] = -c[2];
    if (j < g.ny - 1) row[u + g.nx] = -c[3];
    if (k > 0) row[u - g.nx * g.ny] = -c[4];
    if (k < g.nz - 1) row[u + g.nx * g.ny] = -c[5];
  }
}

// In-place right-looking Cholesky of the dense n x n matrix A (lower triangle
// receives L; the strict upper triangle is zeroed).  One block.  Sets *bad if
// a pivot is not positive.
__global__ void k_cholesky(double* A, int n, int* bad) {
  __shared__ double piv;
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      const double a = A[(i64)j * n + j];
      if (!(a > 0.0)) *bad = 1;
      piv = a > 0.0 ? sqrt(a) : 1.0;
      A[(i64)j * n + j] = piv;
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[(i64)i * n + j] /= piv;
    __syncthreads();
    const i64 m = (i64)(n - j - 1);
    for (i64 t = threadIdx.x; t < m * m; t += blockDim.x) {
      const int ii = j + 1 + (int)(t / m), kk = j + 1 + (int)(t % m);
      if (kk <= ii) A[(i64)ii * n + kk] -= A[(i64)ii * n + j] * A[(i64)kk * n + j];
    }
    __syncthreads();
  }
  for (i64 t = threadIdx.x; t < (i64)n * n; t += blockDim.x)
    if (t % n > t / n) A[t] = 0.0;
}

// Coarsest operator inverse from its Cholesky factor L (n <= 32), row-major,
// for a coarse solve that is one matrix-vector product: Li[0, n*n) receives
// L^-1 (thread c solves L v = e_c by forward substitution, column c) and
// Li[n*n, 2*n*n) the symmetric A^-1 = L^-T L^-1 (entry (l, c) sums
// L^-1(m, l) L^-1(m, c) over m >= max(l, c) in increasing m, so (l, c) and
// (c, l) are the same sum).
__global__ void k_trinv(const double* L, double* Li, int n) {
  const int c = threadIdx.x;
  double* Ai = Li + (i64)n * n;
  if (c < n)
    for (int r = 0; r < n; ++r) {
      double v = 0.0;
      if (r >= c) {
        double s = r == c ? 1.0 : 0.0;
        for (int q = c; q < r; ++q) s -= L[(i64)r * n + q] * Li[(i64)q * n + c];
        v = s / L[(i64)r * n + r];
      }
      Li[(i64)r * n + c] = v;
    }
  __syncthreads();
  if (c < n)
    for (int l = 0; l < n; ++l) {
      double s = 0.0;
      for (int m = l > c ? l : c; m < n; ++m) s = fma(Li[(i64)m * n + l], Li[(i64)m * n + c], s);
      Ai[(i64)l * n + c] = s;
    }
}

// ------------------------------------------------------------ eigenvalue estimate
// Counter-based uniform numbers in [0,1) from Vigna's SplitMix64 finaliser:
// u(seed, stream, idx) = (sm(sm(seed ^ stream << 56) ^ idx) >> 11) * 2^-53.
__host__ __device__ __forceinline__ unsigned long long sm64(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ double u01(unsigned long long seed, unsigned long long stream,
                                               unsigned long long idx) {
  return (double)(sm64(sm64(seed ^ (stream << 56)) ^ idx) >> 11) * (1.0 / 9007199254740992.0);
}

// Start vector of the Lanczos estimate: u - 1/2 at every interior point
// (stream 3, index = interior point number (k ny + j) nx + i); pads stay zero.
template <class TV> __global__ void k_lz_fill(TV* r, Geom g, unsigned long long seed) {
  const i64 n = g.npts();
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.nx), j = (int)((t / g.nx) % g.ny), k = (int)(t / ((i64)g.nx * g.ny));
    r[g.at(i, j, k)] = store_as<TV>(u01(seed, 3, (unsigned long long)t) - 0.5);
  }
}
// z = D^-1 r;  y += a x;  y = x + b y  over whole padded arrays (pads stay zero)
template <class TV> __global__ void k_lz_jacobi(TV* z, const TV* r, const TV* dinv, i64 n) {
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x)
    z[t] = store_as<TV>(cvt<double>(dinv[t]) * cvt<double>(r[t]));
}
template <class TV> __global__ void k_lz_axpy(TV* y, const TV* x, double a, i64 n) {
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x)
    y[t] = store_as<TV>(fma(a, cvt<double>(x[t]), cvt<double>(y[t])));
}
template <class TV> __global__ void k_lz_xpay(TV* y, const TV* x, double b, i64 n) {
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x)
    y[t] = store_as<TV>(fma(b, cvt<double>(y[t]), cvt<double>(x[t])));
}

// ------------------------------------------------------------ scalars
enum FinishMode { FIN_BB = 0, FIN_RR = 1, FIN_RZ0 = 2, FIN_PQ = 3, FIN_RZ = 4, FIN_TRUE = 5 };

// The CG scalar update of a finished reduction (a0, a1) in the given mode.
__device__ __forceinline__ void finish_apply(double a0, double a1, int mode, Scal* s, int flexible) {
  switch (mode) {
    case FIN_BB:
      s->bb = a0;
      s->rr = a0;
      if (!isfinite(a0)) s->status |= 1;
      break;
    case FIN_RR:
      s->rr = a0;
      s->rz_old = a1;
      if (!isfinite(a0)) s->status |= 1;
      break;
    case FIN_TRUE:
      s->true_rr = a0;
      break;
    case FIN_RZ0:
      s->rho = a0;
      s->beta = 0.0;
      if (!isfinite(a0)) s->status |= 1;
      break;
    case FIN_PQ:
      s->pq = a0;
      if (!(a0 > 0.0)) s->status |= isfinite(a0) ? 2 : 1;
      s->alpha = a0 > 0.0 ? s->rho / a0 : 0.0;
      break;
    case FIN_RZ: {
      // Fletcher-Reeves: beta = rho_new / rho.  Polak-Ribiere (flexible):
      // beta = (rho_new - r_new.z_old) / rho.  rho = 0 marks the first
      // iteration of a solve (p = z, beta = 0).
      if (s->rho == 0.0) s->beta = 0.0;
      else s->beta = flexible ? (a0 - s->rz_old) / s->rho : a0 / s->rho;
      s->rho_new = a0;
      s->rho = a0;
      if (!isfinite(a0)) s->status |= 1;
      break;
    }
  }
}

// Fixed-order sum of partials[0..n) (and, with two, of partials[stride ..
// stride+n)) by one block of FIN_THREADS threads: thread t adds elements
// t, t + FIN_THREADS, ... into four accumulators in turn, so that four
// independent loads are in flight per thread, then adds the four in a fixed
// order; the block sum follows.  Only the flexible CG's residual update needs
// the second sum.
constexpr int FIN_THREADS = 256;
__device__ __forceinline__ void fin_sum(const double* part, int n, int stride, bool two, double& a0, double& a1) {
  double s0[4] = {0.0, 0.0, 0.0, 0.0}, s1[4] = {0.0, 0.0, 0.0, 0.0};
  int t = threadIdx.x;
  for (; t + 3 * FIN_THREADS < n; t += 4 * FIN_THREADS) {
#pragma unroll
    for (int u = 0; u < 4; ++u) s0[u] += part[t + u * FIN_THREADS];
    if (two) {
#pragma unroll
      for (int u = 0; u < 4; ++u) s1[u] += part[stride + t + u * FIN_THREADS];
    }
  }
#pragma unroll
  for (int u = 0; u < 3; ++u) {  // at most three elements are left
    const int q = t + u * FIN_THREADS;
    if (q < n) {
      s0[u] += part[q];
      if (two) s1[u] += part[stride + q];
    }
  }
  a0 = (s0[0] + s0[1]) + (s0[2] + s0[3]);
  a1 = (s1[0] + s1[1]) + (s1[2] + s1[3]);
  block_sum2<FIN_THREADS>(a0, a1);
}

// Sums the per-block partials of a reduction and updates the CG scalars.
// With mirror (host memory mapped into the device's address space) the
// updated scalars are also written there, so that the host can read them
// after this kernel without a copy queued on the stream.
__global__ void __launch_bounds__(FIN_THREADS) k_finish(const double* partials, int n, int stride, int mode, Scal* s,
                                                        int flexible, Scal* mirror) {
  pdl_wait();
  double a0, a1;
  fin_sum(partials, n, stride, mode == FIN_RR && flexible, a0, a1);
  if (threadIdx.x == 0) {
    finish_apply(a0, a1, mode, s, flexible);
    if (mirror) {
      *mirror = *s;
      __threadfence_system();
    }
  }
}

// z-slab decomposition: one slab's reduction summed as k_finish sums it, into
// slot[0] and slot[nslab] instead of the scalars ...
__global__ void __launch_bounds__(FIN_THREADS) k_finish_partial(const double* partials, int n, int stride, double* slot,
                                                                int nslab) {
  pdl_wait();
  double a0, a1;
  fin_sum(partials, n, stride, true, a0, a1);
  if (threadIdx.x == 0) {
    slot[0] = a0;
    slot[nslab] = a1;
  }
}

// ... and the slabs' sums added in slab order (the all-reduce of a
// decomposed dot product), then the scalar update.
__global__ void k_combine(const double* slots, int nslab, int mode, Scal* s, int flexible) {
  pdl_wait();
  if (threadIdx.x != 0) return;
  double a0 = 0.0, a1 = 0.0;
  for (int q = 0; q < nslab; ++q) {
    a0 += slots[q];
    a1 += slots[nslab + q];
  }
  finish_apply(a0, a1, mode, s, flexible);
}

// ------------------------------------------------------------ gradient
// dL/dln k_c for every finest cell from phi and lambda (padded float64):
//   sum over the 12 edges e=(p,q) of the cell with an interior end point of
//   -h_a^-2 (lambda_p - lambda_q)(phi_p - phi_q) * dk_e/dln k_c,
//   dk_e/dln k_c = k_e^2/(4 k_c) (harmonic edge mean) or k_c/4 (arithmetic).
__global__ void k_gradient(const double* __restrict__ kc, const double* __restrict__ phi,
                           const double* __restrict__ lam, Geom g, double ihx2, double ihy2, double ihz2,
                           int face_rule, double* __restrict__ grad) {
  const int cx = g.nx + 1, cy = g.ny + 1, cz = g.nz + 1;
  const i64 n = (i64)cx * cy * cz;
  auto cell = [&](int a, int b, int c) { return kc[((i64)c * cy + b) * cx + a]; };
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x) {
    const int ci = (int)(t % cx);
    const i64 r = t / cx;
    const int cj = (int)(r % cy);
    const int ck = (int)(r / cy);
    const double kcv = kc[t];
    double acc = 0.0;
    // corner (a,b,c) of the cell is interior point (ci-1+a, cj-1+b, ck-1+c)
    auto node = [&](const double* v, int a, int b, int c) { return v[g.at(ci - 1 + a, cj - 1 + b, ck - 1 + c)]; };
    auto add = [&](double ke, double ih2, int a0, int b0, int c0, int a1, int b1, int c1) {
      const double dl = node(lam, a0, b0, c0) - node(lam, a1, b1, c1);
      const double dp = node(phi, a0, b0, c0) - node(phi, a1, b1, c1);
      const double dke = face_rule ? 0.25 * kcv : ke * ke / (4.0 * kcv);
      acc += -ih2 * dl * dp * dke;
    };
    for (int v = 0; v < 2; ++v)
      for (int u = 0; u < 2; ++u) {
        {  // x-edge at (J, K) = (cj+u, ck+v): needs J, K interior (full coordinates)
          const int J = cj + u, K = ck + v;
          if (J >= 1 && J <= g.ny && K >= 1 && K <= g.nz) {
            const double ke = edge_mean(cell(ci, J - 1, K - 1), cell(ci, J, K - 1), cell(ci, J - 1, K),
                                        cell(ci, J, K), face_rule);
            add(ke, ihx2, 0, u, v, 1, u, v);
          }
        }
        {  // y-edge at (I, K) = (ci+u, ck+v)
          const int I = ci + u, K = ck + v;
          if (I >= 1 && I <= g.nx && K >= 1 && K <= g.nz) {
            const double ke = edge_mean(cell(I - 1, cj, K - 1), cell(I, cj, K - 1), cell(I - 1, cj, K),
                                        cell(I, cj, K), face_rule);
            add(ke, ihy2, u, 0, v, u, 1, v);
          }
        }
        {  // z-edge at (I, J) = (ci+u, cj+v)
          const int I = ci + u, J = cj + v;
          if (I >= 1 && I <= g.nx && J >= 1 && J <= g.ny) {
            const double ke = edge_mean(cell(I - 1, J - 1, ck), cell(I, J - 1, ck), cell(I - 1, J, ck),
                                        cell(I, J, ck), face_rule);
            add(ke, ihz2, u, v, 0, u, v, 1);
          }
        }
      }
    grad[t] = acc;
  }
}

// ------------------------------------------------------------ telescoped bottom
// The coarse end of the hierarchy runs inside one thread block: levels
// lb..L-1 of the V-cycle (pre-smooth, residual, restriction down; dense
// Cholesky solve on the coarsest level; prolongation and post-smooth up), with
// __syncthreads() between the per-level passes instead of kernel launches.
constexpr int BOT_MAX = 8;
constexpr int BOT_THREADS = 1024;
constexpr int BOT_MAXDEG = 32;  // largest Chebyshev degree

template <class TV, class TC> struct BotLevel {
  Geom g;
  TV* x[2];
  TV* d;
  TV* b;
  TV* r;
  const TV* dinv;
  const TC *kx, *ky, *kz;
  const TC* w;    // Galerkin level: 13 coupling arrays of length g.len (else null)
  const TV* dg;   // and its diagonal
  // Chebyshev constants, rounded to the vector type on the host: a float64
  // to float32 conversion per thread and pass would run on GB300's scarce
  // float64 pipe and dominate the passes of the float32 bottom kernel.
  TV inv_theta;                       // step j = 0: d_0 = s_0 / theta
  TV c1[BOT_MAXDEG], c2[BOT_MAXDEG];  // step j >= 1: d_j = c1[j] d_{j-1} + c2[j] s_j
};

template <class TV, class TC> struct BotArgs {
  BotLevel<TV, TC> lv[BOT_MAX];
  int nlev;            // levels in this kernel; the last one is the coarsest
  int nu_pre, nu_post, degree;
  const double* Lc;    // Cholesky factor of the coarsest operator (n x n)
  const double* Li;    // L^-1, then the operator inverse L^-T L^-1 (n <= 32), else null
  const double* Ac;    // the coarsest operator itself (inexact solve), else null
  double coarse_rtol;  // inexact solve: GMRES-Jacobi to this relative residual,
  int coarse_maxit;    // at most this many steps (<= 32)
  int nc;
};

template <class R, bool CL, class TV, class TC>
__device__ int bot_sweep(const BotLevel<TV, TC>& L, int cur, bool zero, const BotArgs<TV, TC>& a) {
  const R inv_theta = (R)L.inv_theta;
  int j0 = 0;
  if (zero && sizeof(R) == 8 && a.degree > 1) {  // float64: store step 0, then step 1 as an ordinary step
    OpChebStart<R, TV> op{L.b, L.dinv, L.x[cur], L.d, inv_theta};
    block_for<CL>(op, L.g);
    BotSync<CL>::sync();
    zero = false;
    j0 = 1;
  }
  if (zero) {
    if (a.degree == 1) {
      OpChebZero1<R, TV> op{L.b, L.dinv, L.x[cur ^ 1], inv_theta};
      block_for<CL>(op, L.g);
      BotSync<CL>::sync();
      return cur ^ 1;
    }
    TV* dout = a.degree > 2 ? L.d : nullptr;
    if (L.w) {
      OpChebZero27<R, TV, TC> op{L.b, L.dinv, L.x[cur ^ 1], dout, L.w, L.g.len, (R)L.c1[1], (R)L.c2[1], inv_theta};
      block_for<CL>(op, L.g);
    } else {
      OpChebZero<R, TV, TC> op{L.b, L.dinv, L.x[cur ^ 1], dout, L.kx, L.ky, L.kz, (R)L.c1[1], (R)L.c2[1], inv_theta};
      block_for<CL>(op, L.g);
    }
    BotSync<CL>::sync();
    cur ^= 1;
    j0 = 2;
  }
  for (int j = j0; j < a.degree; ++j) {
    const TV* dprev = j > 0 ? L.d : nullptr;
    TV* dout = j + 1 < a.degree ? L.d : nullptr;
    if (L.w) {
      OpChebStep27<R, TV, TC> op{L.x[cur], dprev, L.b, L.dinv, L.x[cur ^ 1], dout, L.w, L.g.len,
                                 (R)L.c1[j], (R)L.c2[j], inv_theta};
      block_for<CL>(op, L.g);
    } else {
      OpChebStep<R, TV, TC> op{L.x[cur], dprev, L.b, L.dinv, L.x[cur ^ 1], dout, L.kx, L.ky, L.kz,
                               (R)L.c1[j], (R)L.c2[j], inv_theta};
      block_for<CL>(op, L.g);
    }
    BotSync<CL>::sync();
    cur ^= 1;
  }
  return cur;
}

// Coarsest solve x = L^-T L^-1 b in float64 with the Cholesky factor.  For
// n <= 32 it is one product with the precomputed inverse (k_trinv): a
// substitution is a chain of n dependent divisions and shuffles, slow on
// GB300's float64 pipe.  Larger n substitute with the whole block.
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Inexact coarsest solve (the truncated coarse solve of the paper's Sec. 5):
// GMRES with the Jacobi preconditioner on the right, classical Gram-Schmidt,
// Givens rotations, from zero, stopped when the rotated residual norm is at
// most rtol ||b|| or after m (<= 32) steps.  Called by all threads of one
// block of at least 32 warps; lane i of a warp holds component i (n <= 32);
// the Krylov basis and the Hessenberg columns live in shared memory.  Per
// step: warps 0-7 form the matrix-vector product from column groups (their
// partial rows added in warp order), warp i forms the Gram-Schmidt
// coefficient of basis vector i (all from the same w), and warp 0 updates w,
// normalises it and (lane 0) applies the rotations.  y holds b on entry and
// x on exit.
__device__ void block_gmres(const double* A, int n, double rtol, int m, double* y) {
  __shared__ double Vs[33 * 32], Hs[33 * 32], gs[33], cs[32], sn[32], ys[32], zs[32], ws[32], part[8 * 32];
  __shared__ double beta_s;
  __shared__ int jj_s, stop_s;
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const bool on = lane < n;
  const double dl = on ? A[lane * n + lane] : 1.0;
  if (wq == 0) {
    const double bi = on ? y[lane] : 0.0;
    const double beta = sqrt(warp_sum_d(bi * bi));
    if (lane == 0) {
      beta_s = beta;
      for (int i = 0; i <= m; ++i) gs[i] = 0.0;
      gs[0] = beta;
      jj_s = 0;
      stop_s = 0;
    }
    if (beta > 0.0) Vs[lane] = bi / beta;
  }
  __syncthreads();
  const double beta = beta_s;
  if (beta > 0.0) {
    for (int j = 0; j < m; ++j) {
      if (wq == 0) zs[lane] = on ? Vs[j * 32 + lane] / dl : 0.0;
      __syncthreads();
      if (wq < 8) {  // w = A z: warp q sums columns q, q + 8, q + 16, q + 24
        double v = 0.0;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const int k = wq + 8 * s;
          if (on && k < n) v = fma(A[lane * n + k], zs[k], v);
        }
        part[wq * 32 + lane] = v;
      }
      __syncthreads();
      if (wq == 0) {
        double w = part[lane];
        for (int q = 1; q < 8; ++q) w += part[q * 32 + lane];
        ws[lane] = on ? w : 0.0;
      }
      __syncthreads();
      if (wq <= j) {  // all coefficients from the same w
        const double h = warp_sum_d(ws[lane] * Vs[wq * 32 + lane]);
        if (lane == 0) Hs[wq * 32 + j] = h;
      }
      __syncthreads();
      if (wq == 0) {
        double w = ws[lane];
        for (int i = 0; i <= j; ++i) w -= Hs[i * 32 + j] * Vs[i * 32 + lane];
        const double hn = sqrt(warp_sum_d(w * w));
        if (hn > 0.0) Vs[(j + 1) * 32 + lane] = w / hn;
        if (lane == 0) {
          Hs[(j + 1) * 32 + j] = hn;
          for (int i = 0; i < j; ++i) {
            const double a = Hs[i * 32 + j], c = Hs[(i + 1) * 32 + j];
            Hs[i * 32 + j] = cs[i] * a + sn[i] * c;
            Hs[(i + 1) * 32 + j] = -sn[i] * a + cs[i] * c;
          }
          const double a = Hs[j * 32 + j], c = Hs[(j + 1) * 32 + j];
          const double d = sqrt(a * a + c * c);
          if (d > 0.0) {
            cs[j] = a / d;
            sn[j] = c / d;
            Hs[j * 32 + j] = d;
            Hs[(j + 1) * 32 + j] = 0.0;
            gs[j + 1] = -sn[j] * gs[j];
            gs[j] = cs[j] * gs[j];
            jj_s = j + 1;
          }
          stop_s = jj_s != j + 1 || fabs(gs[j + 1]) <= rtol * beta || hn == 0.0;
        }
      }
      __syncthreads();
      if (stop_s) break;
    }
    if (threadIdx.x == 0) {  // R y = g
      const int jj = jj_s;
      for (int i = jj - 1; i >= 0; --i) {
        double v = gs[i];
        for (int k = i + 1; k < jj; ++k) v -= Hs[i * 32 + k] * ys[k];
        ys[i] = v / Hs[i * 32 + i];
      }
    }
    __syncthreads();
  }
  if (wq == 0) {
    double xo = 0.0;
    if (beta > 0.0) {
      double sacc = 0.0;
      for (int k = 0; k < jj_s; ++k) sacc += ys[k] * Vs[k * 32 + lane];
      xo = sacc / dl;
    }
    if (on) y[lane] = xo;
  }
  __syncthreads();
}

template <class TV>
__device__ void bot_coarse_solve(const Geom& g, const TV* b, TV* x, const double* Lc, const double* Li, int n,
                                 const double* Ac = nullptr, double crtol = 0.0, int cmaxit = 0) {
  __shared__ double y[1024];
  __shared__ double part[8 * 32];
  for (int u = threadIdx.x; u < n; u += blockDim.x) {
    const int i = u % g.nx, j = (u / g.nx) % g.ny, k = u / (g.nx * g.ny);
    y[u] = cvt<double>(b[g.at(i, j, k)]);
  }
  __syncthreads();
  if (Ac && n <= 32) {
    block_gmres(Ac, n, crtol, cmaxit, y);
  } else if (n <= 32 && Li) {
    // y = A^-1 y with the precomputed symmetric inverse: warp q < 8 sums
    // columns q, q + 8, q + 16, q + 24 (lane w forms row w; its at most four
    // matrix entries are loaded before the first multiply-add, so the
    // chain is one load latency and four float64 FMAs), then thread w adds
    // the eight partial rows in warp order.
    const double* Ai = Li + n * n;
    const int w = threadIdx.x & 31, q = threadIdx.x >> 5;
    double v = 0.0;
    if (q < 8 && w < n) {
      double e[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) e[s] = q + 8 * s < n ? Ai[(q + 8 * s) * n + w] : 0.0;
#pragma unroll
      for (int s = 0; s < 4; ++s)
        if (q + 8 * s < n) v = fma(e[s], y[q + 8 * s], v);
    }
    if (q < 8) part[q * 32 + w] = v;
    __syncthreads();
    if (threadIdx.x < n) {
      double r = part[threadIdx.x];
      for (int u = 1; u < 8; ++u) r += part[u * 32 + threadIdx.x];
      y[threadIdx.x] = r;
    }
  } else {
    for (int c = 0; c < n; ++c) {
      if (threadIdx.x == 0) y[c] /= Lc[(i64)c * n + c];
      __syncthreads();
      for (int i = c + 1 + threadIdx.x; i < n; i += blockDim.x) y[i] -= Lc[(i64)i * n + c] * y[c];
      __syncthreads();
    }
    for (int c = n - 1; c >= 0; --c) {
      if (threadIdx.x == 0) y[c] /= Lc[(i64)c * n + c];
      __syncthreads();
      for (int i = threadIdx.x; i < c; i += blockDim.x) y[i] -= Lc[(i64)c * n + i] * y[c];
      __syncthreads();
    }
  }
  __syncthreads();
  for (int u = threadIdx.x; u < n; u += blockDim.x) {
    const int i = u % g.nx, j = (u / g.nx) % g.ny, k = u / (g.nx * g.ny);
    x[g.at(i, j, k)] = store_as<TV>(y[u]);
  }
  __syncthreads();
}

// L2 prefetch of n bytes at p, one 128-byte line per thread and step
// (threads number tid0 .. tid0 + nthreads - 1)
__device__ __forceinline__ void block_prefetch_l2(const void* p, i64 n, unsigned tid0, unsigned nthreads) {
  if (!p) return;
  for (i64 o = (i64)tid0 * 128; o < n; o += (i64)nthreads * 128)
    asm volatile("prefetch.global.L2 [%0];" ::"l"((const char*)p + o));
}

template <class R, class TV, class TC, bool CL>
__global__ void __launch_bounds__(BOT_THREADS) k_bottom(const __grid_constant__ BotArgs<TV, TC> a) {
  using BS = BotSync<CL>;
  pdl_wait();
  // The streaming passes on the fine levels evict these small arrays from L2
  // between V-cycles: request all of them at once instead of meeting the
  // misses one pass at a time.
  const unsigned tid0 = BS::rank() * blockDim.x + threadIdx.x, nth = BS::blocks() * blockDim.x;
  for (int l = 0; l < a.nlev; ++l) {
    const BotLevel<TV, TC>& V = a.lv[l];
    const i64 nv = V.g.len * (i64)sizeof(TV), nc = V.g.len * (i64)sizeof(TC);
    block_prefetch_l2(V.x[0], nv, tid0, nth);
    block_prefetch_l2(V.x[1], nv, tid0, nth);
    block_prefetch_l2(V.d, nv, tid0, nth);
    block_prefetch_l2(V.b, nv, tid0, nth);
    block_prefetch_l2(V.r, nv, tid0, nth);
    block_prefetch_l2(V.dinv, nv, tid0, nth);
    if (V.w) {
      block_prefetch_l2(V.w, 13 * nc, tid0, nth);
      block_prefetch_l2(V.dg, nv, tid0, nth);
    } else {
      block_prefetch_l2(V.kx, nc, tid0, nth);
      block_prefetch_l2(V.ky, nc, tid0, nth);
      block_prefetch_l2(V.kz, nc, tid0, nth);
    }
  }
  if (a.Li) block_prefetch_l2(a.Li, 2 * (i64)a.nc * a.nc * (i64)sizeof(double), tid0, nth);
  int cur[BOT_MAX];
  const int L = a.nlev;
  for (int l = 0; l < L - 1; ++l) {
    const BotLevel<TV, TC>& V = a.lv[l];
    cur[l] = 0;
    for (int s = 0; s < a.nu_pre; ++s) cur[l] = bot_sweep<R, CL>(V, cur[l], s == 0, a);
    if (a.nu_pre == 0) {
      for (i64 t = tid0; t < V.g.len; t += nth) V.x[0][t] = store_as<TV>(0.0);
      BS::sync();
    }
    if (V.w) {
      OpResidual27<R, TV, TV, TC> res{V.x[cur[l]], V.b, V.r, V.w, V.g.len, V.dg};
      block_for<CL>(res, V.g);
    } else {
      OpResidual<R, TV, TV, TC> res{V.x[cur[l]], V.b, V.r, V.kx, V.ky, V.kz};
      block_for<CL>(res, V.g);
    }
    BS::sync();
    OpRestrict<R, TV> rs{V.g, V.r, a.lv[l + 1].b};
    block_for<CL>(rs, a.lv[l + 1].g);
    BS::sync();
  }
  // the coarsest solve in the first block; its barriers are block-local
  if (BS::rank() == 0)
    bot_coarse_solve<TV>(a.lv[L - 1].g, a.lv[L - 1].b, a.lv[L - 1].x[0], a.Lc, a.Li, a.nc, a.Ac, a.coarse_rtol,
                         a.coarse_maxit);
  BS::sync();
  cur[L - 1] = 0;
  for (int l = L - 2; l >= 0; --l) {
    const BotLevel<TV, TC>& V = a.lv[l];
    OpProlong<R, TV> pr{a.lv[l + 1].g, a.lv[l + 1].x[cur[l + 1]], V.x[cur[l]]};
    block_for<CL>(pr, V.g);
    BS::sync();
    for (int s = 0; s < a.nu_post; ++s) cur[l] = bot_sweep<R, CL>(V, cur[l], false, a);
  }
}

}  // namespace mgdev
