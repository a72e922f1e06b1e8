// Fourth-generation row passes (FP32): the two-step register transforms of
// passes2.cuh, with each tile's input rows brought into shared memory by one
// bulk asynchronous copy (cp.async.bulk, completion counted in bytes on an
// mbarrier).  A tile's rows are contiguous in HBM (X rows of n complex
// values, Y rows of M = 2n), so one instruction moves a whole tile and the
// copy engine, not the threads, generates the addresses.  One staging buffer
// per CTA: as soon as every thread has taken the tile out of it (into
// registers or the exchange tile), the next tile's copy is issued into it and
// runs under the rest of the current tile's work -- the shared memory of a
// second buffer would cost resident warps.
//
// Every wait on an mbarrier is bounded (kWaitLimitCycles).  A CTA whose wait
// gives up ORs kWaitTimeout into jobs.fault, waits (bounded again) for the
// copy it still has in flight and returns; the decision is made CTA-wide
// (__syncthreads_or) so no thread is left at a barrier.
#pragma once
#include "mbar.cuh"
#include "passes2.cuh"

namespace fsa {

// Shared-memory plan of a bulk row pass: the staging buffer of WR input rows
// (ROW complex values each), the exchange tile of the two-step transform, the
// mbarrier.
template <class P, int WR, int ROW> struct BulkGeo {
  static constexpr int NT = WR * P::T;
  static constexpr int PITCH = P::R1 * (P::R2 + 1);
  static constexpr int STG = WR * ROW * 8;
  static constexpr int XCH = WR * PITCH * 8;
  static constexpr int BAR = STG + XCH;  // byte offset of the mbarrier
  static constexpr int SMEM = BAR + 16;
  static_assert(STG % 16 == 0 && BAR % 8 == 0, "staging alignment");
};

// Issue (one thread) the bulk copy of tile `tile` (rows row0.. of its job,
// each ROW complex values) into the staging buffer.
template <int WR, int ROW>
__device__ __forceinline__ void issue_rows(const Jobs& jobs, long long tpj, long long rows, long long tile, float2* dst,
                                           unsigned long long* bar) {
  const Job& jb = jobs.j[tile / tpj];
  const long long row0 = (tile % tpj) * WR;
  const long long nr = rows - row0 < WR ? rows - row0 : WR;
  const unsigned bytes = (unsigned)(nr * ROW * 8);
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(bar, bytes);
  bulk_g2s(dst, static_cast<const float2*>(jb.in) + row0 * ROW, bytes, bar);
}

// After a timeout: record it and drain the copy still in flight.
__device__ __forceinline__ void bulk_abort(const Jobs& jobs, unsigned long long* bar, int it) {
  if (threadIdx.x == 0) {
    if (jobs.fault) atomicOr(jobs.fault, kWaitTimeout);
    mbar_wait(bar, it & 1);
  }
  __syncthreads();
}

template <int WR, int ROW>
__device__ __forceinline__ void bulk_prologue(const Jobs& jobs, long long tpj, long long rows, long long total,
                                              float2* stg, unsigned long long* bar) {
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && blockIdx.x < total) issue_rows<WR, ROW>(jobs, tpj, rows, blockIdx.x, stg, bar);
}

// ------------------------------------------------------------ row forward --
constexpr bool kRowFwdBulkStore = true;
constexpr bool kRowInvBulkStore = true;
// PAD = false: rows of M inputs (the DDI grid reading's unpadded transform).
template <class P, int WR, bool PAD = true>
__global__ void __launch_bounds__(BulkGeo<P, WR, P::M / 2>::NT) k4_row_fwd(const Jobs jobs, long long rows) {
  using V = float2;
  constexpr int M = P::M, n = PAD ? M / 2 : M, R1 = P::R1, R2 = P::R2, T = P::T;
  using G = BulkGeo<P, WR, n>;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* stg = reinterpret_cast<V*>(smraw);
  V* xch = reinterpret_cast<V*>(smraw + G::STG);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smraw + G::BAR);
  const int u = threadIdx.x % T, l = threadIdx.x / T;
  V* line = xch + l * G::PITCH;
  const long long tpj = (rows + WR - 1) / WR;
  const long long total = tpj * jobs.count;
  bulk_prologue<WR, n>(jobs, tpj, rows, total, stg, bar);
  int it = 0;
  for (long long tile = blockIdx.x; tile < total; tile += gridDim.x, ++it) {
    const bool late = !mbar_wait(bar, it & 1);
    const Job& jb = jobs.j[tile / tpj];
    const long long row = (tile % tpj) * WR + l;
    const bool ok = row < rows;
    V* __restrict__ y = static_cast<V*>(jb.out) + row * M;
    const V* src = stg + l * n;
    stepA_fwd<P, V, PAD>(
        u,
        [&](int t, int r) {
          const int p = t + R2 * r;
          return p < n ? src[p] : czero<V>();
        },
        [&](int q, int t, V v) { line[q * (R2 + 1) + t] = v; });
    if (__syncthreads_or(late)) {
      bulk_abort(jobs, bar, it);
      return;
    }
    // every thread is done with the staging buffer: refill it
    if (threadIdx.x == 0 && tile + gridDim.x < total) issue_rows<WR, n>(jobs, tpj, rows, tile + gridDim.x, stg, bar);
    V bv[R2];
#pragma unroll
    for (int t = 0; t < R2; ++t) bv[t] = line[u * (R2 + 1) + t];
    rfft<R2, true>(bv);
    if constexpr (PAD && kRowFwdBulkStore) {
      // the tile's output rows go out by one bulk copy from the exchange
      // tile, rewritten as WR contiguous rows of M values once every thread
      // has taken its step-B inputs out of it
      __syncthreads();
      V* out = xch + l * M;
#pragma unroll
      for (int s = 0; s < R2; ++s) out[u + R1 * s] = bv[s];
      fence_proxy_async_smem();
      __syncthreads();
      if (threadIdx.x == 0) {
        const long long row0 = (tile % tpj) * WR;
        const long long nr = rows - row0 < WR ? rows - row0 : WR;
        bulk_s2g(static_cast<V*>(jb.out) + row0 * M, xch, (unsigned)(nr * M * 8));
        bulk_commit();
        bulk_wait_read0();  // the exchange tile is free again before the barrier below
      }
    } else if (ok) {
#pragma unroll
      for (int s = 0; s < R2; ++s) y[u + R1 * s] = bv[s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) bulk_wait0();
}

// ------------------------------------------------------------ row inverse --
// PAD = false: all M outputs of a row kept.
template <class P, int WR, bool PAD = true>
__global__ void __launch_bounds__(BulkGeo<P, WR, P::M>::NT) k4_row_inv(const Jobs jobs, long long rows) {
  using V = float2;
  constexpr int M = P::M, n = PAD ? M / 2 : M, R1 = P::R1, R2 = P::R2, T = P::T;
  using G = BulkGeo<P, WR, M>;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* stg = reinterpret_cast<V*>(smraw);
  V* xch = reinterpret_cast<V*>(smraw + G::STG);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smraw + G::BAR);
  const int u = threadIdx.x % T, l = threadIdx.x / T;
  V* line = xch + l * G::PITCH;
  const long long tpj = (rows + WR - 1) / WR;
  const long long total = tpj * jobs.count;
  bulk_prologue<WR, M>(jobs, tpj, rows, total, stg, bar);
  int it = 0;
  for (long long tile = blockIdx.x; tile < total; tile += gridDim.x, ++it) {
    const bool late = !mbar_wait(bar, it & 1);
    const Job& jb = jobs.j[tile / tpj];
    const long long row = (tile % tpj) * WR + l;
    const bool ok = row < rows;
    V* __restrict__ x = static_cast<V*>(jb.out) + row * n;
    const V* src = stg + l * M;
    V bv[R2];
#pragma unroll
    for (int s = 0; s < R2; ++s) bv[s] = src[u + R1 * s];
    stepB_inv<P, V>(u, bv, [&](int q, int t, V v) { line[q * (R2 + 1) + t] = v; });
    if (__syncthreads_or(late)) {
      bulk_abort(jobs, bar, it);
      return;
    }
    if (threadIdx.x == 0 && tile + gridDim.x < total) issue_rows<WR, M>(jobs, tpj, rows, tile + gridDim.x, stg, bar);
    constexpr bool STB = PAD && kRowInvBulkStore && R1 % 2 == 0;
    V o[P::PA][R1 / 2];  // STB: this thread's outputs, stored after the barrier
    stepA_inv<P, V, PAD>(
        u, [&](int q, int t) { return line[q * (R2 + 1) + t]; },
        [&](int t, int r, V v) {
          const int p = t + R2 * r;
          if constexpr (STB) {
            o[(t - u) / T][r] = v;
          } else {
            if (p < n && ok) x[p] = v;
          }
        });
    if constexpr (STB) {
      // the tile's output rows (n values each, contiguous in X) leave by one
      // bulk copy from the exchange tile, rewritten as WR rows of n values
      // once every thread has read its step-A inputs out of it
      __syncthreads();
      V* out = xch + l * n;
#pragma unroll
      for (int i = 0; i < P::PA; ++i) {
        const int t = u + T * i;
#pragma unroll
        for (int r = 0; r < R1 / 2; ++r) {
          const int p = t + R2 * r;
          if ((P::PA * T == R2 || t < R2) && p < n) out[p] = o[i][r];
        }
      }
      fence_proxy_async_smem();
      __syncthreads();
      if (threadIdx.x == 0) {
        const long long row0 = (tile % tpj) * WR;
        const long long nr = rows - row0 < WR ? rows - row0 : WR;
        bulk_s2g(static_cast<V*>(jb.out) + row0 * n, xch, (unsigned)(nr * n * 8));
        bulk_commit();
        bulk_wait_read0();  // the exchange tile is free again before the barrier below
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) bulk_wait0();
}

}  // namespace fsa
