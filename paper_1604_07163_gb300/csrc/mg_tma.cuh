// TMA-staged z-marching stencil kernels for the larger levels.
//
// Each block owns a 32 x 8 tile of (i, j) columns and walks planes k0..k1-1.
// Per plane, one thread issues bulk tensor copies (cp.async.bulk.tensor, TMA)
// of every array the step needs into a ring of shared-memory stages:
//   - the stencil vector with a halo of one point in x and y (the x halo is
//     widened to 16 bytes so that every copy starts on a 16-byte boundary);
//   - kx with its -x neighbour column, ky with its -y neighbour row, kz of the
//     plane (the plane below is still resident in the previous stage);
//   - centre-only fields (D^-1, b, d, the float64 CG residual).
// Completion is tracked with one mbarrier per stage (expected transaction
// bytes).  Planes k-1, k, k+1 of the stencil vector are resident while plane
// k is computed, and the copies of plane k+2 are in flight.  Every wait on an
// mbarrier is bounded (poll_limit polls); a block whose wait gives up sets bit
// ST_TIMEOUT of the status word, then waits, with the full TMA_POLL_LIMIT, for
// every copy it has issued whose completion it has not yet seen (the stage
// whose wait gave up included), and returns without writing the rest of its
// outputs.  After ST_TIMEOUT the host must treat the whole solve, and every
// kernel that ran after this one on the stream, as invalid; mg_solve then
// returns MG_ERR_DEVICE_TIMEOUT.  (Should the drain itself give up, copies
// could still land in the shared memory of a block that the SM schedules
// next: one more reason to discard everything after the flag.)
//
// Arrays are viewed as 2-D tensors of rows of Px elements (the padded layout
// of mg_device.cuh puts interior row j of plane k at row
// off/Px + k*Py + j).  Copies that reach outside the tensor read zeros, which
// is the value of the vector pads they stand for.  The one slot a copy cannot
// reach, kx of the edge entering the row from the boundary (stored in the
// last slot of the previous row), is read directly from global memory.
#pragma once
#include <cuda.h>

#include "mg_device.cuh"

namespace mgdev {

constexpr int TT_X = 32, TT_Y = 8, TT_THREADS = 256, TT_NS = 4;
constexpr int ST_TIMEOUT = 4;  // status bit set by a bounded wait that gave up
constexpr int TMA_POLL_LIMIT = 1 << 20;  // polls of one bounded wait (each may suspend briefly)

enum TmaKind { TK_STEP = 0, TK_ZERO = 1, TK_RESID = 2 };

struct TmaMaps {
  CUtensorMap m[8];  // 0 F0, 1 F1, 2 KX, 3 KY, 4 KZ, 5 C0, 6 C1, 7 C2
};

// ---- PTX helpers ------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after limit polls (each poll may suspend the thread
// for a short hardware-defined time; limit 0 gives up at once).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, int limit) {
  for (int it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// ---- shared-memory stage layout ----------------------------------------------
template <class T> struct XHalo {
  static constexpr int XH = 16 / (int)sizeof(T);  // x halo in elements (16 bytes)
  static constexpr int BW = TT_X + 2 * XH;         // box width
};
constexpr int al128(int b) { return (b + 127) / 128 * 128; }

template <int KIND, bool HAS_D, bool DOT, class TV, class TC> struct TmaLayout {
  static constexpr int F0 = 0;                                                       // full-halo vector
  static constexpr int F0B = XHalo<TV>::BW * (TT_Y + 2) * (int)sizeof(TV);
  static constexpr int F1 = al128(F0 + F0B);                                         // second full-halo (ZERO: D^-1)
  static constexpr int F1B = KIND == TK_ZERO ? F0B : 0;
  static constexpr int KX = al128(F1 + F1B);
  static constexpr int KXB = XHalo<TC>::BW * TT_Y * (int)sizeof(TC);
  static constexpr int KY = al128(KX + KXB);
  static constexpr int KYB = TT_X * (TT_Y + 1) * (int)sizeof(TC);
  static constexpr int KZ = al128(KY + KYB);
  static constexpr int KZB = TT_X * TT_Y * (int)sizeof(TC);
  static constexpr int CB = TT_X * TT_Y * (int)sizeof(TV);
  static constexpr int C0 = al128(KZ + KZB);  // STEP: D^-1
  static constexpr int C0B = KIND == TK_STEP ? CB : 0;
  static constexpr int C1 = al128(C0 + C0B);  // STEP, RESID: b
  static constexpr int C1B = KIND != TK_ZERO ? CB : 0;
  static constexpr int C2 = al128(C1 + C1B);  // STEP with d_{j-1}
  static constexpr int C2B = HAS_D ? CB : 0;
  static constexpr int STAGE = al128(C2 + C2B);
  static constexpr int TX_BYTES = F0B + F1B + KXB + KYB + KZB + C0B + C1B + C2B;
  static constexpr int SMEM = TT_NS * STAGE + 128;  // + alignment slack
};

template <class TV, class TC> struct TmaArgs {
  Geom g;
  int kchunk;
  int rowbase;       // off / Px: 2-D row of interior point (0, 0, 0)
  TV* xout;          // STEP, ZERO: new iterate; RESID: residual
  TV* dout;          // direction written for the next step (or null)
  const TC* kx;      // global kx (for the boundary edge entering each row)
  float c1, c2, inv_theta;
  double dc1, dc2, dinv_theta;
  double* partials;  // DOT: per-block sums of b.z (OpChebStepDot)
  int* status;       // bit ST_TIMEOUT on a wait that gave up
  int poll_limit;    // polls of each wait in the main loop (TMA_POLL_LIMIT; 0 only to test the give-up path)
};

template <int KIND, bool HAS_D, bool DOT, class TV, class TC>
__global__ void __launch_bounds__(TT_THREADS) k_tma_stencil(const __grid_constant__ TmaMaps maps,
                                                            const TmaArgs<TV, TC> a) {
  using Lay = TmaLayout<KIND, HAS_D, DOT, TV, TC>;
  using R = TV;
  constexpr int XV = XHalo<TV>::XH, BWV = XHalo<TV>::BW;
  constexpr int XC = XHalo<TC>::XH, BWC = XHalo<TC>::BW;
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t full[TT_NS];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  const Geom& g = a.g;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int i0 = blockIdx.x * TT_X, j0 = blockIdx.y * TT_Y;
  const int k0 = blockIdx.z * a.kchunk;
  const int k1 = min(k0 + a.kchunk, g.nz);
  const int i = i0 + tx, j = j0 + ty;
  const bool active = i < g.nx && j < g.ny;
  const R c1 = (R)(sizeof(R) == 8 ? a.dc1 : a.c1), c2 = (R)(sizeof(R) == 8 ? a.dc2 : a.c2);
  const R inv_theta = (R)(sizeof(R) == 8 ? a.dinv_theta : a.inv_theta);

  auto stage = [&](int s) { return smem + s * Lay::STAGE; };
  pdl_wait();
  if (tid == 0) {
    for (int s = 0; s < TT_NS; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  // copies for sequence number n (plane k0 - 1 + n) into stage n % NS
  const int nload = (k1 - k0) + 2;
  auto issue = [&](int n) {
    const int s = n % TT_NS;
    unsigned char* st = stage(s);
    const int row = a.rowbase + (k0 - 1 + n) * g.Py + j0;
    mbar_expect_tx(&full[s], Lay::TX_BYTES);
    tma_load_2d(st + Lay::F0, &maps.m[0], i0 - XV, row - 1, &full[s]);
    if constexpr (KIND == TK_ZERO) tma_load_2d(st + Lay::F1, &maps.m[1], i0 - XV, row - 1, &full[s]);
    tma_load_2d(st + Lay::KX, &maps.m[2], i0 - XC, row, &full[s]);
    tma_load_2d(st + Lay::KY, &maps.m[3], i0, row - 1, &full[s]);
    tma_load_2d(st + Lay::KZ, &maps.m[4], i0, row, &full[s]);
    if constexpr (KIND == TK_STEP) tma_load_2d(st + Lay::C0, &maps.m[5], i0, row, &full[s]);
    if constexpr (KIND != TK_ZERO) tma_load_2d(st + Lay::C1, &maps.m[6], i0, row, &full[s]);
    if constexpr (HAS_D) tma_load_2d(st + Lay::C2, &maps.m[7], i0, row, &full[s]);
  };
  int issued = 0;
  if (tid == 0) {
    for (int n = 0; n < TT_NS && n < nload; ++n) issue(n);
    issued = TT_NS < nload ? TT_NS : nload;
  }

  double acc = 0.0, acc1 = 0.0;
  bool bad = false;
  int done = -1;  // every sequence number <= done has been seen complete by this thread
  for (int k = k0; k < k1; ++k) {
    const int n = k - k0 + 1;
    for (int m = done + 1; m <= n + 1; ++m) {
      if (!mbar_wait_bounded(&full[m % TT_NS], (unsigned)((m / TT_NS) & 1), a.poll_limit)) {
        bad = true;
        break;
      }
      done = m;
    }
    if (__syncthreads_or(bad)) {  // every thread leaves together
      bad = true;
      break;
    }
    const unsigned char* S = stage(n % TT_NS);
    const unsigned char* Sm = stage((n - 1) % TT_NS);
    const unsigned char* Sp = stage((n + 1) % TT_NS);
    if (active) {
      const int p = (int)g.at(i, j, k);
      // coefficients
      const TC* KXs = (const TC*)(S + Lay::KX);
      const TC* KYs = (const TC*)(S + Lay::KY);
      const R cxm = (i == 0) ? cvt<R>(__ldg(a.kx + p - 1)) : cvt<R>(KXs[ty * BWC + tx + XC - 1]);
      const R cxp = cvt<R>(KXs[ty * BWC + tx + XC]);
      const R cym = cvt<R>(KYs[ty * TT_X + tx]);
      const R cyp = cvt<R>(KYs[(ty + 1) * TT_X + tx]);
      const R czm = cvt<R>(((const TC*)(Sm + Lay::KZ))[ty * TT_X + tx]);
      const R czp = cvt<R>(((const TC*)(S + Lay::KZ))[ty * TT_X + tx]);
      const int c = (ty + 1) * BWV + tx + XV;  // centre in a full-halo tile
      auto F = [&](const unsigned char* st, int off) -> R {
        if constexpr (KIND == TK_ZERO) {
          // x_1 = D^-1 b / theta formed from the two staged fields
          return inv_theta * (cvt<R>(((const TV*)(st + Lay::F1))[off]) * cvt<R>(((const TV*)(st + Lay::F0))[off]));
        } else {
          return cvt<R>(((const TV*)(st + Lay::F0))[off]);
        }
      };
      R Ssum = cxm * F(S, c - 1);
      Ssum = fma(cxp, F(S, c + 1), Ssum);
      Ssum = fma(cym, F(S, c - BWV), Ssum);
      Ssum = fma(cyp, F(S, c + BWV), Ssum);
      Ssum = fma(czm, F(Sm, c), Ssum);
      Ssum = fma(czp, F(Sp, c), Ssum);
      const int cc = ty * TT_X + tx;  // centre in a centre-only tile
      const R u = F(S, c);
      if constexpr (KIND == TK_RESID) {
        const R D = ((cxm + cxp) + (cym + cyp)) + (czm + czp);
        const R b = cvt<R>(((const TV*)(S + Lay::C1))[cc]);
        const R rv = (b + Ssum) - D * u;
        a.xout[p] = store_as<TV>(rv);
      } else {
        R dinv, b;
        if constexpr (KIND == TK_ZERO) {
          dinv = cvt<R>(((const TV*)(S + Lay::F1))[c]);
          b = cvt<R>(((const TV*)(S + Lay::F0))[c]);
        } else {
          dinv = cvt<R>(((const TV*)(S + Lay::C0))[cc]);
          b = cvt<R>(((const TV*)(S + Lay::C1))[cc]);
        }
        const R s = fma(dinv, b + Ssum, -u);
        R dn;
        if constexpr (KIND == TK_ZERO) dn = fma(c1, u, c2 * s);  // d_0 = x_1
        else if constexpr (HAS_D) dn = fma(c1, cvt<R>(((const TV*)(S + Lay::C2))[cc]), c2 * s);
        else dn = s * inv_theta;
        const R xn = u + dn;
        a.xout[p] = store_as<TV>(xn);
        if (a.dout) a.dout[p] = store_as<TV>(dn);
        if constexpr (DOT) acc = fma(to_double(((const TV*)(S + Lay::C1))[cc]), to_double(store_as<TV>(xn)), acc);
      }
    }
    __syncthreads();
    // the stage of plane k-1 is free: copy plane k - 1 + NS into it
    if (tid == 0 && issued < nload) {
      fence_proxy_async();
      issue(issued);
      ++issued;
    }
  }
  pdl_trigger();
  if (bad) {
    // thread 0 issued every copy; stages reuse only after all threads passed
    // their waits, so each sequence number in (done, issued) is the pending
    // phase of its stage
    if (tid == 0) {
      atomicOr(a.status, ST_TIMEOUT);
      for (int m = done + 1; m < issued; ++m)
        mbar_wait_bounded(&full[m % TT_NS], (unsigned)((m / TT_NS) & 1), TMA_POLL_LIMIT);
    }
    return;
  }
  if constexpr (DOT) {
    block_sum2<TT_THREADS>(acc, acc1);
    if (tid == 0) a.partials[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = acc;
  }
}

}  // namespace mgdev
