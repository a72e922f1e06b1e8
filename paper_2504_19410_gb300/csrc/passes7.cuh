// Seventh-generation FP32 passes: the row-forward (axis 2), middle (axis 1,
// with the spectrum multiply) and row-inverse (axis 2) passes of a solve as
// ONE persistent kernel whose CTAs take their work from a dispenser.
//
// Those three passes depend on each other plane by plane only: the middle
// pass of axis-0 frequency plane k0 needs the row-forward output of that
// plane (all n1 rows of Y[k0]), and the row inverse of the plane needs its
// middle pass.  The work items are tiles of 16 rows (row passes) or 16
// columns (middle pass) of one plane.  They are handed out by one atomic
// counter in a fixed order -- the row-forward tiles of plane s, the middle
// tiles of plane s - L and the row-inverse tiles of plane s - 2L, for
// s = 0, 1, ... ("slots") -- so that
//   * a CTA that takes an item waits only for items handed out before it,
//     to CTAs that are already running: the wait always ends (no deadlock,
//     whatever the number of resident CTAs);
//   * with the lag L larger than the items in flight, the wait is normally
//     already over when the item is taken;
//   * the planes between the row forward and the row inverse (2L planes of Y,
//     a few MB) stay in the 129 MB L2, so Y is written to HBM once (when its
//     dirty lines are evicted) instead of being written, read, written and
//     read again by three separate kernels;
//   * the HBM-latency-bound row tiles run on the SMs at the same time as the
//     arithmetic-bound middle tiles.
//
// Completion: after an item, every thread's stores are ordered before the
// item's counter increment (barrier, then one thread's fence and atomic add,
// the pattern of a grid-wide barrier); a CTA that depends on the counter
// polls it with acquire loads (one thread), then a barrier, and reads the
// data through L2 only (ld.global.cg), since the L1 of its SM is not coherent
// with the other SMs' stores.  Every wait is bounded (kWaitLimitCycles): a
// CTA whose wait gives up ORs kWaitTimeout into jobs.fault and stops taking
// work, so the kernel always returns.
//
// Counters (job 0's Job::aux, 4-byte words, zeroed by the launcher before the
// launch): [0] the dispenser, then per plane q of the launch (q = job * K0 +
// k0) [2 + 2q] finished row-forward items and [3 + 2q] finished middle items.
#pragma once
#include "mbar.cuh"
#include "passes2.cuh"

namespace fsa {

// Shared memory of a CTA: the exchange tile of the two-step transforms (row
// or column layout), a staging area that receives the NEXT item's inputs
// while the current one computes (row forward: one bulk copy of its W input
// rows; middle: per-thread cp.async copies in the generation-3 layout; the
// row inverse reads its inputs directly), the mbarrier of the bulk copies.
template <class P> struct Geo7 {
  static constexpr int W = Geo2<P>::W;  // rows or columns per item
  static constexpr int NT = Geo2<P>::NT;
  static constexpr int XCH = Geo2<P>::SM_ROWS > Geo2<P>::SM_STRIDED ? Geo2<P>::SM_ROWS : Geo2<P>::SM_STRIDED;
  static constexpr int STG_ROW = W * (P::M / 2) * 8;
  static constexpr int STG = Stage2<P>::BYTES > STG_ROW ? Stage2<P>::BYTES : STG_ROW;
  static constexpr int BAR = XCH + STG;
  static constexpr int SMEM = BAR + 16;
  static_assert(XCH % 16 == 0 && STG % 16 == 0, "staging alignment");
};

// The dispenser's order.  a, b, c: items per plane of the row forward, the
// middle and the row inverse; NP planes; lag L (1 <= L, 2 L <= NP).  Slots
// 0..L-1 hold row-forward items only, L..2L-1 row forward and middle,
// 2L..NP-1 all three kinds, NP..NP+L-1 middle and row inverse, the last L
// row inverse only; p0..p3 are the item indices where those ranges end.
// Item counts stay below 2^31 (checked by the launcher).
struct PipeSched {
  int a, b, c, NP, L;
  int p0, p1, p2, p3, total;
};

inline PipeSched make_pipe_sched(int a, int b, int c, int NP, int L) {
  PipeSched s;
  s.a = a;
  s.b = b;
  s.c = c;
  s.NP = NP;
  s.L = L;
  s.p0 = L * a;
  s.p1 = s.p0 + L * (a + b);
  s.p2 = s.p1 + (NP - 2 * L) * (a + b + c);
  s.p3 = s.p2 + L * (b + c);
  s.total = s.p3 + L * c;
  return s;
}

// item -> kind (0 row forward, 1 middle, 2 row inverse), plane, tile
__host__ __device__ inline void pipe_decode(const PipeSched& s, int i, int& kind, int& plane, int& tile) {
  int slot, k;
  bool rf = false, mid = false;  // whether the slot's range holds row-forward / middle items
  if (i < s.p0) {
    slot = i / s.a, k = i % s.a, rf = true;
  } else if (i < s.p1) {
    slot = s.L + (i - s.p0) / (s.a + s.b), k = (i - s.p0) % (s.a + s.b), rf = mid = true;
  } else if (i < s.p2) {
    slot = 2 * s.L + (i - s.p1) / (s.a + s.b + s.c), k = (i - s.p1) % (s.a + s.b + s.c), rf = mid = true;
  } else if (i < s.p3) {
    slot = s.NP + (i - s.p2) / (s.b + s.c), k = (i - s.p2) % (s.b + s.c), mid = true;
  } else {
    slot = s.NP + s.L + (i - s.p3) / s.c, k = (i - s.p3) % s.c;
  }
  if (rf && k < s.a) {
    kind = 0, plane = slot, tile = k;
    return;
  }
  if (rf) k -= s.a;
  if (mid && k < s.b) {
    kind = 1, plane = slot - s.L, tile = k;
    return;
  }
  if (mid) k -= s.b;
  kind = 2, plane = slot - 2 * s.L, tile = k;
}

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// release add: this thread's earlier writes, and those ordered before them
// (a CTA barrier), are visible before the counter moves
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

// true once *c >= need; false after kWaitLimitCycles SM clock cycles
__device__ __forceinline__ bool wait_count(const unsigned* c, unsigned need) {
  if (ld_acquire_u32(c) >= need) return true;
  const long long t0 = clock64();
  while (ld_acquire_u32(c) < need) {
    __nanosleep(64);
    if (clock64() - t0 > kWaitLimitCycles) return false;
  }
  return true;
}

// The counter an item waits for and the count it needs (kind 0: none).
__device__ __forceinline__ const unsigned* pipe_dep(const unsigned* ctr, const PipeSched& sc, int kind, int plane,
                                                    unsigned& need) {
  need = kind == 1 ? (unsigned)sc.a : (unsigned)sc.b;
  return ctr + 2 + 2 * plane + (kind - 1);
}

// Axes: n1 rows of n = M/2 values per plane, middle transform length
// M1 = 2 n1 = M (this generation needs n1 = n2), K0 planes per job.
template <class P>
__global__ void __launch_bounds__(Geo7<P>::NT, 2) k7_pipe(const Jobs jobs, int n1, int K0, const PipeSched sc) {
  using V = float2;
  using G = Geo7<P>;
  constexpr int M = P::M, n = M / 2, W = G::W, R1 = P::R1, R2 = P::R2, T = P::T, NT = G::NT;
  constexpr int PITCH = Geo2<P>::PITCH, RA = Stage2<P>::RA;
  extern __shared__ __align__(16) unsigned char smraw[];
  // the items: two slots, the current item's and the next one's (index,
  // kind, plane, tile, flags: bit 0 its dependency is met, bit 1 its inputs
  // are staged); thread 0 fills the next slot before the current item's
  // exchange barrier, so the CTA goes on to the next item without another
  // barrier whenever that item is ready
  __shared__ int s_item[2][5];
  V* sm = reinterpret_cast<V*>(smraw);
  V* stg = reinterpret_cast<V*>(smraw + G::XCH);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smraw + G::BAR);
  unsigned* ctr = static_cast<unsigned*>(const_cast<void*>(jobs.j[0].aux));
  const int tid = threadIdx.x;
  // thread mappings: rows (u = sub-transform index, l = row of the tile) and
  // middle (l = column of the tile, u paired with its mirror in one warp)
  const int ur = tid % T, lr = tid / T;
  const int lm = tid % W, um = mid_u<P>(tid);
  int fills = 0;  // bulk copies issued into the staging area (mbarrier phase)
  // thread 0's queue: the next item and the one after it
  int q_nxt = 0, q_nxt2 = 0;
  // thread 0: the finished item whose completion is not signalled yet (its
  // counter word, or null).  The signal -- a fence, which waits until the
  // item's stores have reached L2, then the count -- is sent at the next
  // item's exchange barrier, when those stores are long done, instead of
  // holding the CTA right after the item
  unsigned* pend = nullptr;
  auto signal = [&]() {
    if (pend) {
      __threadfence();
      atomicAdd(pend, 1u);
      pend = nullptr;
    }
  };

  // the staging of item (kind, plane, tile)'s inputs: rows by one bulk copy
  // (thread 0), middle columns by every thread's cp.async of its own elements
  auto stage = [&](int kind, int plane, int tile) {
    const Job& jb = jobs.j[plane / K0];
    const int k0 = plane % K0;
    if (kind == 0) {
      if (tid == 0) {
        const int j0 = tile * W;
        const int nr = n1 - j0 < W ? n1 - j0 : W;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar, (unsigned)(nr * n * 8));
        bulk_g2s(stg, static_cast<const V*>(jb.in) + ((long long)k0 * n1 + j0) * n, (unsigned)(nr * n * 8), bar);
      }
    } else {
      const V* col = static_cast<const V*>(jb.out) + (long long)k0 * n * M + tile * W + lm;
#pragma unroll
      for (int i = 0; i < P::PA; ++i) {
#pragma unroll
        for (int r = 0; r < RA; ++r) {
          const int t = um + T * i;
          const int p = t + R2 * r;
          const bool live = t < R2 && p < n;
          cp_async8(&stg[((i * RA + r) * T + um) * W + lm], live ? col + (long long)p * M : col, live ? 8 : 0);
        }
      }
      cp_async_commit();
    }
  };

  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    const int cur = (int)atomicAdd(ctr, 1u);
    q_nxt = (int)atomicAdd(ctr, 1u);
    int kind = -1, plane = 0, tile = 0;
    if (cur < sc.total) {
      pipe_decode(sc, cur, kind, plane, tile);
      unsigned need;
      if (kind > 0 && !wait_count(pipe_dep(ctr, sc, kind, plane, need), need)) {
        if (jobs.fault) atomicOr(jobs.fault, kWaitTimeout);
        kind = -1;
      }
    }
    s_item[0][0] = cur, s_item[0][1] = kind, s_item[0][2] = plane, s_item[0][3] = tile, s_item[0][4] = 1;
  }
  __syncthreads();
  for (int buf = 0;; buf ^= 1) {
    const int kind = s_item[buf][1], plane = s_item[buf][2], tile = s_item[buf][3];
    const bool staged = s_item[buf][4] & 2;
    if (kind < 0) break;
    int* nx = s_item[buf ^ 1];
    const int job = plane / K0, k0 = plane % K0;
    const Job& jb = jobs.j[job];
    // thread 0: the item after next (used an item later), and the next one's
    // dependency (used at the exchange barrier)
    unsigned dep_v = 0, dep_need = 0;
    int nk = -1, npl = 0, nt = 0;
    if (tid == 0) {
      q_nxt2 = (int)atomicAdd(ctr, 1u);
      if (q_nxt < sc.total) {
        pipe_decode(sc, q_nxt, nk, npl, nt);
        // relaxed: this thread's item loads must not wait for it; the fence
        // below makes it an acquire once it is seen to be met
        if (nk > 0) dep_v = ld_relaxed_u32(pipe_dep(ctr, sc, nk, npl, dep_need));
      }
    }
    // thread 0, just before the item's exchange barrier: the next slot, with
    // its inputs staged now if its dependency is already met (the row
    // inverse reads its inputs directly)
    auto decide = [&]() {
      if (tid == 0) {
        const bool ready = nk < 0 || nk == 0 || dep_v >= dep_need;
        if (ready && nk > 0) __threadfence();
        nx[0] = q_nxt, nx[1] = nk, nx[2] = npl, nx[3] = nt;
        nx[4] = (ready ? 1 : 0) | (ready && (nk == 0 || nk == 1) ? 2 : 0);
      }
    };
    auto prefetch = [&]() {
      if (nx[4] & 2) {
        stage(nx[1], nx[2], nx[3]);
        if (nx[1] == 0) ++fills;
      }
    };
    if (kind == 0) {  // row forward: X rows -> Y rows (pad n -> M, transform)
      const int j = tile * W + lr;
      const bool ok = j < n1;
      const long long row = (long long)k0 * n1 + j;
      V* __restrict__ y = static_cast<V*>(jb.out) + row * M;
      V* line = sm + lr * PITCH;
      if (staged) {
        const bool late = !mbar_wait(bar, (fills - 1) & 1);
        if (__syncthreads_or(late)) {
          if (tid == 0) {
            if (jobs.fault) atomicOr(jobs.fault, kWaitTimeout);
            mbar_wait(bar, (fills - 1) & 1);  // the copy still in flight
          }
          break;
        }
        const V* src = stg + lr * n;
        stepA_fwd<P, V, true>(
            ur,
            [&](int t, int r) {
              const int p = t + R2 * r;
              return (p < n && ok) ? src[p] : czero<V>();
            },
            [&](int q, int t, V v) { line[q * (R2 + 1) + t] = v; });
      } else {
        const V* __restrict__ x = static_cast<const V*>(jb.in) + row * n;
        stepA_fwd<P, V, true>(
            ur,
            [&](int t, int r) {
              const int p = t + R2 * r;
              return (p < n && ok) ? x[p] : czero<V>();
            },
            [&](int q, int t, V v) { line[q * (R2 + 1) + t] = v; });
      }
      decide();
      __syncthreads();
      if (tid == 0) signal();
      prefetch();
      V b[R2];
#pragma unroll
      for (int t = 0; t < R2; ++t) b[t] = line[ur * (R2 + 1) + t];
      rfft<R2, true>(b);
      if (ok) {
#pragma unroll
        for (int s = 0; s < R2; ++s) y[ur + R1 * s] = b[s];
      }
    } else if (kind == 1) {  // middle: Y columns in place, times the spectrum
      const int k2 = tile * W + lm;
      V* __restrict__ col = static_cast<V*>(jb.out) + (long long)k0 * n * M + k2;
      const float* __restrict__ srow =
          static_cast<const float*>(jb.S) + (long long)k0 * (n + 1) * (n + 1) + min(k2, M - k2);
      if (staged) {
        cp_async_wait_all();
        stepA_fwd<P, V, true>(
            um,
            [&](int t, int r) {
              const int i = (t - um) / T;
              return r < RA ? stg[((i * RA + r) * T + um) * W + lm] : czero<V>();
            },
            [&](int q, int t, V v) { sm[(q * R2 + t) * W + lm] = v; });
      } else {
        stepA_fwd<P, V, true>(
            um,
            [&](int t, int r) {
              const int p = t + R2 * r;
              return p < n ? __ldcg(col + (long long)p * M) : czero<V>();
            },
            [&](int q, int t, V v) { sm[(q * R2 + t) * W + lm] = v; });
      }
      decide();
      __syncthreads();
      if (tid == 0) signal();
      prefetch();
      MidSpec<P> sp;
      mid_load<P>(sp, srow, um, true, n + 1);
      V b[R2];
#pragma unroll
      for (int t = 0; t < R2; ++t) b[t] = sm[(um * R2 + t) * W + lm];
      rfft<R2, true>(b);
      mid_multiply<P, kMulSpectrum>(b, sp, um, jb, k0, k2, M, true);
      stepB_inv<P, V>(um, b, [&](int q, int t, V v) { sm[(q * R2 + t) * W + lm] = v; });
      __syncthreads();
      stepA_inv<P, V, true>(
          um, [&](int q, int t) { return sm[(q * R2 + t) * W + lm]; },
          [&](int t, int r, V v) {
            const int p = t + R2 * r;
            if (p < n) col[(long long)p * M] = v;
          });
    } else {  // row inverse: Y rows -> X rows (transform, crop M -> n)
      const int j = tile * W + lr;
      const bool ok = j < n1;
      const long long row = (long long)k0 * n1 + j;
      const V* __restrict__ y = static_cast<const V*>(jb.out) + row * M;
      V* __restrict__ x = static_cast<V*>(const_cast<void*>(jb.in)) + row * n;
      V* line = sm + lr * PITCH;
      V b[R2];
#pragma unroll
      for (int s = 0; s < R2; ++s) b[s] = ok ? __ldcg(y + ur + R1 * s) : czero<V>();
      stepB_inv<P, V>(ur, b, [&](int q, int t, V v) { line[q * (R2 + 1) + t] = v; });
      decide();
      __syncthreads();
      if (tid == 0) signal();
      prefetch();
      stepA_inv<P, V, true>(
          ur, [&](int q, int t) { return line[q * (R2 + 1) + t]; },
          [&](int t, int r, V v) {
            const int p = t + R2 * r;
            if (p < n && ok) x[p] = v;
          });
    }
    __syncthreads();  // the item's stores are done, its shared memory is free
    // thread 0: the item's completion is pending (every thread's stores are
    // ordered before its signal by this barrier); only if the next item's
    // dependency was not met yet, the signal goes now and the CTA waits at a
    // barrier for the dependency (which may be this very item)
    if (tid == 0 && kind < 2) pend = ctr + 2 + 2 * plane + kind;
    if (!(nx[4] & 1)) {
      if (tid == 0) {
        signal();
        unsigned need;
        if (!wait_count(pipe_dep(ctr, sc, nx[1], nx[2], need), need)) {
          if (jobs.fault) atomicOr(jobs.fault, kWaitTimeout);
          nx[1] = -1;
        }
      }
      __syncthreads();
    }
    if (tid == 0) q_nxt = q_nxt2;
  }
  if (tid == 0) signal();
  // nothing may land in shared memory after the CTA exits
  cp_async_wait_all();
}

}  // namespace fsa
