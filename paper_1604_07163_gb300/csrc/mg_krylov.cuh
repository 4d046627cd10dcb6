// Vector kernels of the flexible GMRES outer iteration (Saad, Iterative
// Methods for Sparse Linear Systems, Alg. 9.6; the paper's outer Krylov
// method in Sec. 5).  All arithmetic is float64; the preconditioned vectors
// z_j are kept in the V-cycle's precision.  Every reduction is a fixed tree
// (per-thread sums, block sums in index order, then partials in index order),
// so results repeat bit for bit.
#pragma once
#include "mg_device.cuh"

namespace mgdev {

constexpr int KR_THREADS = 256;
constexpr int KR_MAXV = 8;    // vectors per multi-dot launch
constexpr int KR_MAXC = 264;  // coefficients of one k_maxpy launch (at most the restart length + 1)

// partials[v * nblocks + block] = sum over this block's elements of w . V_v,
// for the NV <= KR_MAXV vectors V_v = V0 + v * vst.  The pass is bound by
// load latency unless each thread keeps enough loads in flight: a thread
// takes 2U consecutive elements per step (U = 8 / NV pairs), issues all of the
// step's 16-byte loads of w and of every V_v, then its multiply-adds.
template <int NV>
__global__ void __launch_bounds__(KR_THREADS) k_mdot(const double* __restrict__ w, const double* __restrict__ V0,
                                                     i64 vst, i64 n, double* partials) {
  constexpr int U = KR_MAXV / NV;  // element pairs per thread and step
  double acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.0;
  const i64 step = 2 * U * (i64)gridDim.x * KR_THREADS;
  i64 t0 = 2 * U * (blockIdx.x * (i64)KR_THREADS) + 2 * threadIdx.x;
  for (; t0 + 2 * (U - 1) * KR_THREADS < n; t0 += step) {  // all U pairs in range
    double2 wt[U], x[U][NV];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const i64 t = t0 + 2 * u * KR_THREADS;
      wt[u] = __ldg(reinterpret_cast<const double2*>(w + t));
#pragma unroll
      for (int v = 0; v < NV; ++v) x[u][v] = __ldg(reinterpret_cast<const double2*>(V0 + v * vst + t));
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] = fma(wt[u].y, x[u][v].y, fma(wt[u].x, x[u][v].x, acc[v]));
  }
  for (int u = 0; u < U; ++u) {  // the last, partial step
    const i64 t = t0 + 2 * u * KR_THREADS;
    if (t < n) {
      const double2 wt = __ldg(reinterpret_cast<const double2*>(w + t));
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double2 x = __ldg(reinterpret_cast<const double2*>(V0 + v * vst + t));
        acc[v] = fma(wt.y, x.y, fma(wt.x, x.x, acc[v]));
      }
    }
  }
#pragma unroll
  for (int v = 0; v < NV; v += 2) {
    double a = acc[v], b = v + 1 < NV ? acc[v + 1] : 0.0;
    block_sum2<KR_THREADS>(a, b);
    if (threadIdx.x == 0) {
      partials[(i64)v * gridDim.x + blockIdx.x] = a;
      if (v + 1 < NV) partials[(i64)(v + 1) * gridDim.x + blockIdx.x] = b;
    }
  }
}

// out[v] = sum of partials[v * nblocks + 0 .. nblocks-1]; one block per vector
__global__ void __launch_bounds__(KR_THREADS) k_mdot_finish(const double* partials, int nblocks, double* out) {
  double a = 0.0, b = 0.0;
  const double* p = partials + (i64)blockIdx.x * nblocks;
  for (int t = threadIdx.x; t < nblocks; t += KR_THREADS) a += p[t];
  block_sum2<KR_THREADS>(a, b);
  if (threadIdx.x == 0) out[blockIdx.x] = a;
}

// y[t] -= sum_v c[v] X_v[t] (NEG: Gram-Schmidt update of w) or
// y[t] += sum_v c[v] X_v[t] (x += Z c at the end of a cycle), for the nv <=
// KR_MAXC vectors X_v = X0 + v * xst; float X_v are widened on the integer
// pipe.  Each thread updates two consecutive elements per step with 16-byte
// (8-byte) accesses and issues the loads of four vectors before their
// multiply-adds; each element still takes its terms in vector order, so the
// result is that of one fma per vector in turn.  The coefficients are read
// once into shared memory.  With RED the block sums of y.y after the update
// go to partials[block] (the norm of the new Arnoldi vector).
template <class TX> __device__ __forceinline__ void ld2d(const TX* a, double& v0, double& v1);
template <> __device__ __forceinline__ void ld2d<double>(const double* a, double& v0, double& v1) {
  const double2 t = __ldg(reinterpret_cast<const double2*>(a));
  v0 = t.x;
  v1 = t.y;
}
template <> __device__ __forceinline__ void ld2d<float>(const float* a, double& v0, double& v1) {
  const float2 t = __ldg(reinterpret_cast<const float2*>(a));
  v0 = f2d_bits(t.x);
  v1 = f2d_bits(t.y);
}
template <class TX, bool NEG, bool RED>
__global__ void __launch_bounds__(KR_THREADS) k_maxpy(double* __restrict__ y, const TX* __restrict__ X0, i64 xst, int nv,
                                                      const double* c, i64 n, double* partials) {
  __shared__ double cs[KR_MAXC];
  for (int v = threadIdx.x; v < nv; v += KR_THREADS) cs[v] = NEG ? -c[v] : c[v];
  __syncthreads();
  double acc = 0.0;
  for (i64 t = 2 * (blockIdx.x * (i64)KR_THREADS + threadIdx.x); t < n; t += 2 * (i64)gridDim.x * KR_THREADS) {
    const double2 y2 = *reinterpret_cast<const double2*>(y + t);
    double a0 = y2.x, a1 = y2.y;
    int v = 0;
    for (; v + 4 <= nv; v += 4) {
      double x0[4], x1[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) ld2d<TX>(X0 + (v + u) * xst + t, x0[u], x1[u]);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a0 = fma(cs[v + u], x0[u], a0);
        a1 = fma(cs[v + u], x1[u], a1);
      }
    }
    for (; v < nv; ++v) {
      double x0, x1;
      ld2d<TX>(X0 + v * xst + t, x0, x1);
      a0 = fma(cs[v], x0, a0);
      a1 = fma(cs[v], x1, a1);
    }
    *reinterpret_cast<double2*>(y + t) = make_double2(a0, a1);
    if constexpr (RED) {
      acc = fma(a0, a0, acc);
      acc = fma(a1, a1, acc);
    }
  }
  if constexpr (RED) {
    double b = 0.0;
    block_sum2<KR_THREADS>(acc, b);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
  }
}

// dst = s * src: a normalised Arnoldi vector (s = 1 / its norm)
__global__ void k_scale(double* __restrict__ dst, const double* __restrict__ src, double s, i64 n) {
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x)
    dst[t] = src[t] * s;
}

// a[t * stride] *= s for t < n, in place: the host-requested data
// perturbations that exercise the error paths (mg_params.test_inject)
__global__ void k_scale_strided(double* a, double s, i64 n, i64 stride) {
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x)
    a[t * stride] *= s;
}

// y = A u in float64 for an operand u stored in the V-cycle precision TZ,
// with the stored float64 diagonal dg (the sum of the six edge coefficients
// in stencil()'s order): y = dg u - S.  Summing the diagonal again would
// cost five more float64 additions per point on GB300's float64 pipe, which
// bounds this kernel.
template <class TZ> struct OpApplyTo64 {
  using Real = double;
  const TZ* u;
  double* y;
  const double* dg;
  const double *kx, *ky, *kz;
  __device__ void prepare() {}
  template <bool NC> __device__ __forceinline__ void pt(const Geom& g, int, int, int, int p, double&, double&) const {
    double D;
    Ld lu{u};
    const double S = stencil<NC, double>(g, p, lu, kx, ky, kz, D);
    y[p] = fma(ldp<NC>(dg + p), lu(p), -S);
  }
  struct Ld {  // float operands widened on the integer pipe
    const TZ* a;
    __device__ __forceinline__ double operator()(int q) const { return to_double(__ldg(a + q)); }
  };
};

}  // namespace mgdev
