// Fifth-generation FP32 outer passes: the pad + R2C along axis 0 and the
// forward axis-2 transform fused into one kernel (rho -> Y), and the inverse
// axis-2 transform and the C2R along axis 0 + crop fused into one (Y -> phi),
// so the half spectrum X of the five-pass schedule never goes to HBM: per
// 256^3 FP32 solve that is 135 MB written and read back twice.
//
// The two axes of a pair meet in an i1-slab (all i0, all i2 for one i1),
// whose X part is (n0 + 1) x n2 complex values (526 KB at n = 256): more than
// one SM's shared memory, so a thread-block cluster of CS CTAs holds it in
// distributed shared memory.  Forward, per slab:
//   phase 1: CTA r transforms its CW = n2 / CS real columns along axis 0
//            (column pairs packed as one complex line, as in passes2.cuh) and
//            stores each output row k0 straight into the shared memory of the
//            CTA that owns that row (st.shared::cluster);
//   cluster barrier (release / acquire: the remote stores are visible);
//   phase 2: CTA r transforms its rows along axis 2 from its own shared
//            memory and writes them to Y;
//   cluster barrier (the rows are consumed before the next slab's stores).
// The inverse runs the same two phases the other way round (rows of Y ->
// columns of X in the owners' shared memory -> C2R along axis 0 -> phi).
//
// Rows k0 = 0 and k0 = n0 of X are real for real rho (the DFT of a real column
// at frequency 0 and M0/2), so they travel as one complex line
// X[0] + i X[n0] ("line 0"): n0 lines of n2 values per slab, n0 / CS per CTA,
// every CTA of the cluster the same work.  Forward, line 0's transform Z is
// split by Hermitian symmetry, Y[0] = (Z[k] + conj Z[-k]) / 2 and
// Y[n0] = (Z[k] - conj Z[-k]) / 2i, with Z[-k] taken from the mirror thread of
// the same line by a warp shuffle; inverse, Y[0] + i Y[n0] transforms to
// X[0] + i X[n0] directly (the rows of Y at k0 = 0 and n0 are Hermitian in k2:
// they are spectra of real sequences).
//
// Every CTA of a cluster runs the same slab loop (slab = cluster index +
// k x cluster count) and the same rounds, so every barrier is reached by all
// threads of the cluster; there are no waits on flags or mbarriers.
//
// The pair moves fewer HBM bytes but the same transform work, with fewer
// resident warps (a slab's share of shared memory per CTA, and only as many
// clusters as the GPCs can place), so whether it beats the separate passes
// depends on the size and the chip: the tuner times both (plan.cu).
#pragma once
#include "mbar.cuh"
#include "passes2.cuh"

namespace fsa {

// ---------------------------------------------- cluster / DSMEM helpers --
__device__ __forceinline__ unsigned cluster_ctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// The shared::cluster address of the same offset in CTA `rank`'s shared memory.
__device__ __forceinline__ unsigned dsmem_map(unsigned smem_addr, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void dsmem_st(unsigned addr, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void dsmem_st(unsigned addr, float4 v) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w)
               : "memory");
}
// All threads of all CTAs of the cluster; orders the shared-memory stores
// before it (local and remote) before the loads after it.
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// The same rendezvous without the release (no memory fence): for the
// barriers that only keep the next slab's remote stores behind this slab's
// reads, whose values are consumed before the arrive.
__device__ __forceinline__ void cluster_rendezvous() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
}

// Tile plan of a fused pair: P0 the axis-0 plan (M0 = 2 n0), P2 the axis-2
// plan (M2 = 2 n2), CS CTAs per cluster, NT threads per CTA.
template <class P0, class P2, int CS, int NT> struct FusedGeo {
  static constexpr int n0 = P0::M / 2, n2 = P2::M / 2, K0 = n0 + 1;
  static constexpr int CW = n2 / CS;   // real columns of one CTA (axis-0 phase)
  static constexpr int LW = CW / 2;    // their complex lines (column pairs)
  static constexpr int W0 = NT / P0::T;  // axis-0 lines per round
  static constexpr int R0 = LW / W0;     // axis-0 rounds
  static constexpr int LR = n0 / CS;     // axis-2 lines of one CTA
  static constexpr int W2 = NT / P2::T;  // axis-2 lines per round
  static constexpr int RR = LR / W2;     // axis-2 rounds
  static constexpr int PITCH2 = P2::R1 * (P2::R2 + 1);
  static constexpr int XCH = (P0::M * W0 > W2 * PITCH2 ? P0::M * W0 : W2 * PITCH2) * 8;
  static constexpr int RCV_F = LR * n2 * 8;  // forward: this CTA's rows, n2 values each
  static constexpr int RCV_I = K0 * CW * 8;  // inverse: this CTA's columns, all K0 rows
  static constexpr int SMEM_F = RCV_F + XCH;
  static constexpr int SMEM_I = RCV_I + XCH;
  static_assert(NT % P0::T == 0 && NT % P2::T == 0, "whole lines per round");
  static_assert(32 % P2::T == 0, "an axis-2 line within one warp (mirror shuffle)");
  static_assert(n2 % (2 * CS) == 0 && LW % W0 == 0 && R0 >= 1, "axis-0 columns split evenly");
  static_assert(n0 % CS == 0 && LR % W2 == 0 && RR >= 1, "axis-2 lines split evenly");
  static_assert(RCV_F % 16 == 0 && RCV_I % 16 == 0, "exchange tile alignment");
};

// --------------------------------------------------------- forward pair --
// jobs.j[i]: in = rho (n0 x n1 x n2 reals), out = Y ((n0+1) x n1 x M2 complex).
template <class P0, class P2, int CS, int NT>
__global__ void __launch_bounds__(NT) k5_fwd(const Jobs jobs, int n1) {
  using V = float2;
  using G = FusedGeo<P0, P2, CS, NT>;
  constexpr int M0 = P0::M, n0 = M0 / 2, M2 = P2::M, n2 = M2 / 2;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* rcv = reinterpret_cast<V*>(smraw);             // [LR][n2]: rows k0 = rank + CS j
  V* xch = reinterpret_cast<V*>(smraw + G::RCV_F);  // exchange tile of the two-step transforms
  const unsigned rank = cluster_ctarank();
  const unsigned rcv_addr = smem_u32(rcv);
  const long long C = (long long)n1 * n2;
  const long long total = (long long)n1 * jobs.count;
  const long long nclusters = gridDim.x / CS;
  cluster_rendezvous();  // the whole cluster is running before the first remote store
  for (long long slab = blockIdx.x / CS; slab < total; slab += nclusters) {
    const Job& jb = jobs.j[slab / n1];
    const int i1 = (int)(slab % n1);
    // phase 1: pad + R2C along axis 0 of columns i2 in [rank CW, (rank + 1) CW)
    {
      constexpr int W = G::W0, R1 = P0::R1, R2 = P0::R2;
      const float* __restrict__ rho = static_cast<const float*>(jb.in);
      const int l = threadIdx.x % W, u = threadIdx.x / W;
#pragma unroll 1
      for (int rd = 0; rd < G::R0; ++rd) {
        const int i2 = (int)rank * G::CW + 2 * (rd * W + l);  // this lane's column pair (i2, i2 + 1)
        const long long c = (long long)i1 * n2 + i2;
        stepA_fwd<P0, V, true>(
            u,
            [&](int t, int r) {
              const int p = t + R2 * r;
              return p < n0 ? *reinterpret_cast<const V*>(rho + (long long)p * C + c) : czero<V>();
            },
            [&](int q, int t, V v) { xch[(q * R2 + t) * W + l] = v; });
        __syncthreads();
        V b[R2];
#pragma unroll
        for (int t = 0; t < R2; ++t) b[t] = xch[(u * R2 + t) * W + l];
        rfft<R2, true>(b);
        __syncthreads();
#pragma unroll
        for (int s = 0; s < R2; ++s) xch[(u + R1 * s) * W + l] = b[s];
        __syncthreads();
        // Z = DFT(a + i b) of the pair: A[k] = (Z[k] + conj Z[M0-k]) / 2,
        // B[k] = (Z[k] - conj Z[M0-k]) / 2i; k = 0 carries line 0 (k = n0 too)
        for (int k = u; k < n0; k += P0::T) {
          const V zk = xch[k * W + l];
          float4 v;
          if (k == 0) {
            const V zh = xch[n0 * W + l];  // Z[M0/2]: A[n0] = Re, B[n0] = Im
            v = make_float4(zk.x, zh.x, zk.y, zh.y);
          } else {
            const V zm = xch[(M0 - k) * W + l];
            v = make_float4(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y), 0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
          }
          // row k lives in CTA k % CS as its local row k / CS
          dsmem_st(dsmem_map(rcv_addr + (unsigned)(((k / CS) * n2 + i2) * 8), (unsigned)(k % CS)), v);
        }
        __syncthreads();  // the exchange tile is rewritten by the next round
      }
    }
    cluster_barrier();  // every row of the slab has arrived
    // phase 2: forward axis-2 transform of rows k0 = rank + CS j, j < LR
    {
      constexpr int W = G::W2, R1 = P2::R1, R2 = P2::R2, T = P2::T;
      V* __restrict__ Y = static_cast<V*>(jb.out);
      const int u = threadIdx.x % T, l = threadIdx.x / T;
      V* line = xch + l * G::PITCH2;
#pragma unroll 1
      for (int rd = 0; rd < G::RR; ++rd) {
        const int j = rd * W + l;
        const int k0 = (int)rank + CS * j;  // 0: line 0 (rows 0 and n0)
        const V* src = rcv + j * n2;
        stepA_fwd<P2, V, true>(
            u,
            [&](int t, int r) {
              const int p = t + R2 * r;
              return p < n2 ? src[p] : czero<V>();
            },
            [&](int q, int t, V v) { line[q * (R2 + 1) + t] = v; });
        __syncthreads();
        V bv[R2];
#pragma unroll
        for (int t = 0; t < R2; ++t) bv[t] = line[u * (R2 + 1) + t];
        rfft<R2, true>(bv);
        // bv[s] = Z[k2], k2 = u + R1 s
        V* __restrict__ y = Y + ((long long)k0 * n1 + i1) * M2;
        if (rank == 0 && rd == 0 && threadIdx.x < 32) {  // the warp holding line 0 (warp-uniform)
          // Z[M2 - k2]: thread (R1 - u) % R1 of the same line, element R2 - 1 - s
          // (u > 0) or this thread's own element (R2 - s) % R2 (u = 0)
          const int lane = threadIdx.x & 31;
          const int src_lane = (lane & ~(T - 1)) | ((T - u) % T);
          V* __restrict__ yn = Y + ((long long)n0 * n1 + i1) * M2;
#pragma unroll
          for (int s = 0; s < R2; ++s) {
            V m;
            m.x = __shfl_sync(0xffffffffu, bv[R2 - 1 - s].x, src_lane);
            m.y = __shfl_sync(0xffffffffu, bv[R2 - 1 - s].y, src_lane);
            if (u == 0) m = bv[(R2 - s) % R2];
            const V z = bv[s];
            if (k0 == 0) {
              y[u + R1 * s] = mk(0.5f * (z.x + m.x), 0.5f * (z.y - m.y));
              yn[u + R1 * s] = mk(0.5f * (z.y + m.y), 0.5f * (m.x - z.x));
            } else {
              y[u + R1 * s] = z;
            }
          }
        } else {
#pragma unroll
          for (int s = 0; s < R2; ++s) y[u + R1 * s] = bv[s];
        }
        __syncthreads();
      }
    }
    cluster_rendezvous();  // the rows are consumed before the next slab's phase 1
  }
}

// --------------------------------------------------------- inverse pair --
// jobs.j[i]: in = Y ((n0+1) x n1 x M2 complex), out = phi (n0 x n1 x n2 reals).
template <class P0, class P2, int CS, int NT>
__global__ void __launch_bounds__(NT) k5_inv(const Jobs jobs, int n1) {
  using V = float2;
  using G = FusedGeo<P0, P2, CS, NT>;
  constexpr int M0 = P0::M, n0 = M0 / 2, M2 = P2::M, n2 = M2 / 2, CW = G::CW;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* rcv = reinterpret_cast<V*>(smraw);             // [K0][CW]: X of this CTA's columns
  V* xch = reinterpret_cast<V*>(smraw + G::RCV_I);
  const unsigned rank = cluster_ctarank();
  const unsigned rcv_addr = smem_u32(rcv);
  const long long C = (long long)n1 * n2;
  const long long total = (long long)n1 * jobs.count;
  const long long nclusters = gridDim.x / CS;
  cluster_rendezvous();
  for (long long slab = blockIdx.x / CS; slab < total; slab += nclusters) {
    const Job& jb = jobs.j[slab / n1];
    const int i1 = (int)(slab % n1);
    // phase A: inverse axis-2 transform of rows k0 = rank + CS j (crop to
    // i2 < n2), each value stored to the CTA owning column i2
    {
      constexpr int W = G::W2, R1 = P2::R1, R2 = P2::R2, T = P2::T;
      const V* __restrict__ Y = static_cast<const V*>(jb.in);
      const int u = threadIdx.x % T, l = threadIdx.x / T;
      V* line = xch + l * G::PITCH2;
#pragma unroll 1
      for (int rd = 0; rd < G::RR; ++rd) {
        const int j = rd * W + l;
        const int k0 = (int)rank + CS * j;
        const V* __restrict__ y = Y + ((long long)k0 * n1 + i1) * M2;
        V bv[R2];
        if (k0 == 0) {  // line 0: Y[0] + i Y[n0]
          const V* __restrict__ yn = Y + ((long long)n0 * n1 + i1) * M2;
#pragma unroll
          for (int s = 0; s < R2; ++s) {
            const V a = y[u + R1 * s], b = yn[u + R1 * s];
            bv[s] = mk(a.x - b.y, a.y + b.x);
          }
        } else {
#pragma unroll
          for (int s = 0; s < R2; ++s) bv[s] = y[u + R1 * s];
        }
        stepB_inv<P2, V>(u, bv, [&](int q, int t, V v) { line[q * (R2 + 1) + t] = v; });
        __syncthreads();
        stepA_inv<P2, V, true>(
            u, [&](int q, int t) { return line[q * (R2 + 1) + t]; },
            [&](int t, int r, V v) {
              const int p = t + R2 * r;
              if (p < n2) {
                const unsigned owner = (unsigned)(p / CW);
                const int cl = p % CW;
                if (k0 == 0) {  // v = X[0] + i X[n0], both real
                  dsmem_st(dsmem_map(rcv_addr + (unsigned)(cl * 8), owner), mk(v.x, 0.f));
                  dsmem_st(dsmem_map(rcv_addr + (unsigned)((n0 * CW + cl) * 8), owner), mk(v.y, 0.f));
                } else {
                  dsmem_st(dsmem_map(rcv_addr + (unsigned)((k0 * CW + cl) * 8), owner), v);
                }
              }
            });
        __syncthreads();
      }
    }
    cluster_barrier();  // this CTA's columns are complete
    // phase B: C2R along axis 0 of columns i2 in [rank CW, (rank + 1) CW), crop to i0 < n0
    {
      constexpr int W = G::W0, R1 = P0::R1, R2 = P0::R2;
      float* __restrict__ phi = static_cast<float*>(jb.out);
      const int l = threadIdx.x % W, u = threadIdx.x / W;
#pragma unroll 1
      for (int rd = 0; rd < G::R0; ++rd) {
        const int cl = 2 * (rd * W + l);  // local column pair (cl, cl + 1)
        const long long c = (long long)i1 * n2 + (long long)rank * CW + cl;
        // Z[k] = A[k] + i B[k] with A, B Hermitian: k > n0 from M0 - k
        V b[R2];
#pragma unroll
        for (int s = 0; s < R2; ++s) {
          const int k = u + R1 * s;
          const bool lo = k <= n0;
          const float4 ab = *reinterpret_cast<const float4*>(rcv + (lo ? k : M0 - k) * CW + cl);
          b[s] = lo ? mk(ab.x - ab.w, ab.y + ab.z) : mk(ab.x + ab.w, ab.z - ab.y);
        }
        stepB_inv<P0, V>(u, b, [&](int q, int t, V v) { xch[(q * R2 + t) * W + l] = v; });
        __syncthreads();
        stepA_inv<P0, V, true>(
            u, [&](int q, int t) { return xch[(q * R2 + t) * W + l]; },
            [&](int t, int r, V v) {
              const int p = t + R2 * r;
              if (p < n0) *reinterpret_cast<V*>(phi + (long long)p * C + c) = v;
            });
        __syncthreads();
      }
    }
    cluster_rendezvous();  // the columns are consumed before the next slab's phase A
  }
}

}  // namespace fsa
