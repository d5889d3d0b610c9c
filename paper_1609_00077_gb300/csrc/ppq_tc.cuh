// Quartic (T9) topology on the 5th-generation tensor cores (tcgen05, sm_103a).
//
//   r2[Y,Z][o] += 1/2 sum_{X,W} s Cl[X,Y][c1] Cl[X,Z][c2] G[X,W][g] Cl[W,Y][c3] Cl[W,Z][c4]
//
// Rows are the unordered pairs p = (Y < Z), packed 128 to a tile.  For every
// distinct link pair (c1, c2) the row-wise (Khatri-Rao) operand
//   A[p][X] = Cl[X,Y][c1] Cl[X,Z][c2]
// is generated in shared memory and multiplied by B_g[W][X] = G[X,W][g] for
// the g of that pair, D[p][W] = sum_X A[p][X] B_g[W][X], with the
// accumulator in tensor memory (TMEM).  The W contraction against
// Cl[W,Y][c3] Cl[W,Z][c4] is the epilogue: one thread per row reads its row of
// D from TMEM.
//
// FP32 accuracy from TF32 inputs: each operand is split x = hi + lo with hi,
// lo TF32-rounded, and D accumulates hi*hi + hi*lo + lo*hi (three MMAs per
// K step); the dropped lo*lo term is below 2^-22 relative.
//
// Shared-memory operands use the no-swizzle K-major canonical layout: 8-row x
// 16-byte core matrices, K-adjacent cores 128 B apart (leading byte offset),
// 8-row groups 256 B apart (stride byte offset); one K stage is 8 TF32 values.
//
// Roles (800 threads): warps 0-15 epilogue (TMEM lane quarter = warp % 4; the
// four warps of a quarter take the channels of output o = warp / 4 mod 4, so
// every (row, o) sum has one owner and a fixed order; D is read from TMEM
// eight columns at a time next to the loads of the Cl factors), warps 16-23
// producers (A generation, two threads per row, each one 4-wide K core of a
// stage; thread 512 also issues the bulk copies of B and of the Cl slices),
// warp 24 TMEM allocation and MMA issue (lane 0).
// Each CTA writes the sums of its rows (all 29 outputs) to its own slot of
// a partial buffer, part[slot][p][o]; k_t9_reduce adds the slots in a fixed
// order, so the result does not depend on scheduling.
// Every wait is bounded; on a timeout the CTA stops issuing work, lets its
// copies and MMAs drain (again bounded), flags the error and writes a NaN into
// its slot so that the residual reads as non-finite.
#pragma once
#include <cstdint>

namespace ppq {
namespace tc {

constexpr int kStages = 4;
constexpr int kRows = 128;                 // MMA M, rows per tile
constexpr int kMaxCols = 256;              // TMEM columns per accumulator buffer
constexpr int kEpiThreads = 512;           // warps 0-15
constexpr int kProdThreads = 256;          // warps 16-23: two per row, one K core (4 of the 8 K) each
constexpr int kProdBase = kEpiThreads;
constexpr int kProdWarp0 = kProdBase / 32;
constexpr int kMmaWarp = kProdWarp0 + kProdThreads / 32;
constexpr int kThreads = (kMmaWarp + 1) * 32;
static_assert(kEpiThreads % kRows == 0 && kEpiThreads / kRows == 4, "four epilogue groups of 128 rows");
static_assert(kProdThreads == 2 * kRows, "two producer threads per row");
static_assert(kThreads == 800, "24 role warps + the MMA warp");
constexpr long long kWaitCycles = 2000000000LL;  // about 1 s at 2 GHz
constexpr int kChunkFields = 12;           // c1, c2, n_g, n_cols, g[4], q[4]

__device__ __forceinline__ uint32_t su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(su32(b))
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(su32(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait for completion of the phase with the given parity; false on timeout or abort
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort) {
  if (mbar_try(b, parity)) return true;
  long long t0 = clock64();
  while (true) {
    if (mbar_try(b, parity)) return true;
    if (*abort) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort = 1;
      return false;
    }
  }
}
// the same, ignoring the abort flag (used to drain in-flight work)
__device__ __forceinline__ bool mbar_drain(uint64_t* b, uint32_t parity) {
  long long t0 = clock64();
  while (!mbar_try(b, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   su32(dst)),
               "l"(src), "r"(bytes), "r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// smem matrix descriptor: start, leading / stride byte offsets, fixed 0b001 at
// bits 46-48, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  constexpr uint64_t lbo = 128, sbo = 256;
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) | (1ull << 46);
}
// instruction descriptor, kind::tf32: D F32 (bits 4-5 = 1), A and B TF32
// (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28
__device__ __forceinline__ uint32_t idesc_tf32(int n_cols) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n_cols >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}
// 16 consecutive TMEM columns of this thread's lane, waited on before return
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
// 8 consecutive TMEM columns of this thread's lane, issued without waiting:
// the registers are valid after tmem_wait8 on the same array
__device__ __forceinline__ void tmem_issue8(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
// wait for the issued TMEM loads; the registers pass through the wait so that
// no use of them is scheduled before it
__device__ __forceinline__ void tmem_wait8(uint32_t* r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])
               :
               : "memory");
}
// 4 consecutive TMEM columns of this thread's lane, waited on before return
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float* v) {
  uint32_t r[4];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// B operands, split and laid out per K stage:
// bpre[g][split][kc][W / 8][kcore][W % 8][k % 4], X = 8 kc + 4 kcore + k % 4,
// value G[X,W][g] (zero outside X, W < N); W runs over Npad = 16 ceil(N / 16)
__global__ void k_t9_bprep(int N, int Npad, int Kc, const float* __restrict__ pg, float* __restrict__ bpre) {
  size_t per = (size_t)Npad * 8;                       // floats per (g, split, kc) block
  size_t tot = (size_t)PPQ_NS36 * Kc * per;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= tot) return;
  size_t off = i % per;
  size_t gk = i / per;
  int kc = (int)(gk % Kc), g = (int)(gk / Kc);
  int e = (int)(off & 3), r8 = (int)((off >> 2) & 7), kcore = (int)((off >> 5) & 1), rg = (int)(off >> 6);
  int W = rg * 8 + r8, X = kc * 8 + kcore * 4 + e;
  float v = (W < N && X < N) ? pg[((size_t)X * N + W) * PPQ_NS36 + g] : 0.f;
  float hi = tf32_rna(v), lo = tf32_rna(v - hi);
  bpre[((size_t)(g * 2 + 0) * Kc + kc) * per + off] = hi;
  bpre[((size_t)(g * 2 + 1) * Kc + kc) * per + off] = lo;
}

// dynamic shared memory map (byte offsets)
struct Smem {
  static constexpr size_t kA = (size_t)kRows * 8 * 4;      // one split of one A stage
  static constexpr size_t kB = (size_t)kMaxCols * 8 * 4;   // one split of one B stage
  static constexpr size_t kStageBytes = 2 * kA + 2 * kB;
  static constexpr int kNBars = 4 * kStages + 9;
  static size_t __host__ __device__ slices() { return (size_t)kStages * kStageBytes; }
  static size_t __host__ __device__ t9(int NNp) { return slices() + 2 * 2 * (size_t)NNp * 4; }
  static size_t __host__ __device__ rows(int NNp) { return t9(NNp) + (size_t)kRows * PPQ_NA2 * 4; }
  static size_t __host__ __device__ bars(int NNp) { return rows(NNp) + (size_t)kRows * 2 * 4; }
  static size_t __host__ __device__ total(int NNp) { return bars(NNp) + kNBars * 8 + 16; }
};

// One CTA per (row tile, range of chunks); a chunk is one (c1, c2) with up to
// four of its g (n_cols = n_g Npad TMEM columns).  cta[3 b] = tile, first, end;
// every tile has nslot CTAs, in order, and CTA b writes slot b % nslot.
template <int NW>
__global__ void __launch_bounds__(kThreads, 1)
    k_t9_tc(int N, int P, int Kc, int NNp, const float* __restrict__ clT, const float* __restrict__ bpre,
            const int* __restrict__ cta, const int16_t* __restrict__ chunks, int nslot,
            float* __restrict__ part, int* __restrict__ err) {
  constexpr int Npad = NW;
  extern __shared__ __align__(1024) unsigned char sm[];
  float* sA = reinterpret_cast<float*>(sm);                              // [S][2][128 x 8]
  float* sB = reinterpret_cast<float*>(sm + kStages * 2 * Smem::kA);     // [S][2][256 x 8]
  float* sCl = reinterpret_cast<float*>(sm + Smem::slices());            // [2][2][NNp]
  float* st9 = reinterpret_cast<float*>(sm + Smem::t9(NNp));             // [128][29]
  int* rowYZ = reinterpret_cast<int*>(sm + Smem::rows(NNp));             // [128][2]
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + Smem::bars(NNp));
  uint64_t* fullA = bars;                     // [S] producers wrote A (count 256)
  uint64_t* fullB = bars + kStages;           // [S] B copies landed (count 1 + tx)
  uint64_t* empty = bars + 2 * kStages;       // [S] MMAs of the stage done (commit)
  uint64_t* done = bars + 3 * kStages;        // all MMAs of the CTA done (commit)
  uint64_t* slf = bars + 4 * kStages;         // [2] Cl slices landed (count 1 + tx)
  uint64_t* sle = slf + 2;                    // [2] producers done with the slices (count 256)
  uint64_t* tmf = sle + 2;                    // [2] accumulator buffer ready (commit)
  uint64_t* tme = tmf + 2;                    // [2] epilogue done with the buffer (count 512)
  uint32_t* tbase = reinterpret_cast<uint32_t*>(bars + Smem::kNBars);
  volatile int* abort = reinterpret_cast<volatile int*>(tbase + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = cta[3 * blockIdx.x], cb = cta[3 * blockIdx.x + 1], ce = cta[3 * blockIdx.x + 2];
  const int nloc = ce - cb;
  const size_t blk = (size_t)Npad * 8;        // floats of one (g, split, kc) block of bpre

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&fullA[s], kProdThreads);
      mbar_init(&fullB[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&slf[b], 1);
      mbar_init(&sle[b], kProdThreads);
      mbar_init(&tmf[b], 1);
      mbar_init(&tme[b], kEpiThreads);
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < kRows) {
    int p = tile * kRows + tid, Y = -1, Z = -1;
    if (p < P) {
      int rem = p;
      Y = 0;
      while (rem >= N - 1 - Y) { rem -= N - 1 - Y; ++Y; }
      Z = Y + 1 + rem;
    }
    rowYZ[2 * tid] = Y;
    rowYZ[2 * tid + 1] = Z;
  }
  if (tid < kRows)
    for (int o = 0; o < PPQ_NA2; ++o) st9[tid * PPQ_NA2 + o] = 0.f;
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tbase)),
                 "r"(2 * kMaxCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_before();
  }
  __syncthreads();
  tc_after();
  const uint32_t tmem = *tbase;

  if (warp >= kProdWarp0 && warp < kMmaWarp) {
    // ------------------------------------------------------------ producers
    const int pr = tid - kProdBase, r = pr & (kRows - 1), hh = pr / kRows;  // row, K core
    const int Y = rowYZ[2 * r], Z = rowYZ[2 * r + 1];
    const bool lead = (pr == 0);
    int issued_b = 0, issued_s = 0;  // stage / slice fills issued by the lead thread
    if (lead && nloc > 0) {
      const int16_t* h = chunks + (size_t)cb * kChunkFields;
      mbar_arrive_tx(&slf[0], 2u * NNp * 4);
      bulk_g2s(sCl, clT + (size_t)h[0] * NNp, NNp * 4, &slf[0]);
      bulk_g2s(sCl + NNp, clT + (size_t)h[1] * NNp, NNp * 4, &slf[0]);
      issued_s = 1;
    }
    int it = 0;
    for (int l = 0; l < nloc && !*abort; ++l) {
      const int16_t* h = chunks + (size_t)(cb + l) * kChunkFields;
      const int ng = h[2];
      const int b = l & 1;
      if (lead && l + 1 < nloc) {
        // prefetch the next chunk's slices once every producer is done with chunk l - 1
        if (l >= 1 && !mbar_wait(&sle[b ^ 1], ((l - 1) >> 1) & 1, abort)) break;
        const int16_t* hn = h + kChunkFields;
        float* dst = sCl + (size_t)(b ^ 1) * 2 * NNp;
        mbar_arrive_tx(&slf[b ^ 1], 2u * NNp * 4);
        bulk_g2s(dst, clT + (size_t)hn[0] * NNp, NNp * 4, &slf[b ^ 1]);
        bulk_g2s(dst + NNp, clT + (size_t)hn[1] * NNp, NNp * 4, &slf[b ^ 1]);
        ++issued_s;
      }
      if (!mbar_wait(&slf[b], (l >> 1) & 1, abort)) break;
      const float* c1s = sCl + (size_t)b * 2 * NNp;
      const float* c2s = c1s + NNp;
      for (int kc = 0; kc < Kc; ++kc, ++it) {
        const int s = it % kStages;
        const uint32_t ph = (it / kStages) & 1;
        if (!mbar_wait(&empty[s], ph ^ 1, abort)) break;
        float* bdst = sB + (size_t)s * 2 * (Smem::kB / 4);
        if (lead) {
          mbar_arrive_tx(&fullB[s], (uint32_t)(ng * 2 * blk * 4));
          for (int j = 0; j < ng; ++j)
            for (int sp = 0; sp < 2; ++sp)
              bulk_g2s(bdst + sp * (Smem::kB / 4) + j * blk,
                       bpre + ((size_t)(h[4 + j] * 2 + sp) * Kc + kc) * blk, (uint32_t)(blk * 4), &fullB[s]);
          ++issued_b;
        }
        float hi[4], lo[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          int X = kc * 8 + 4 * hh + k;
          float a = (Y >= 0 && X < N) ? c1s[X * N + Y] * c2s[X * N + Z] : 0.f;
          hi[k] = tf32_rna(a);
          lo[k] = tf32_rna(a - hi[k]);
        }
        float* adst = sA + (size_t)s * 2 * (Smem::kA / 4);
        const int base = (r >> 3) * 64 + (r & 7) * 4 + hh * 32;   // floats: row group 256 B, row 16 B, K core
        *reinterpret_cast<float4*>(adst + base) = make_float4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<float4*>(adst + (Smem::kA / 4) + base) = make_float4(lo[0], lo[1], lo[2], lo[3]);
        fence_async_smem();
        mbar_arrive(&fullA[s]);
      }
      mbar_arrive(&sle[b]);
    }
    if (lead) {
      // let every issued copy land before the CTA can exit
      for (int k = (issued_b > kStages ? issued_b - kStages : 0); k < issued_b; ++k)
        mbar_drain(&fullB[k % kStages], (k / kStages) & 1);
      for (int k = (issued_s > 2 ? issued_s - 2 : 0); k < issued_s; ++k) mbar_drain(&slf[k & 1], (k >> 1) & 1);
    }
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      int it = 0;
      for (int l = 0; l < nloc && !*abort; ++l) {
        const int16_t* h = chunks + (size_t)(cb + l) * kChunkFields;
        const int ncols = h[3];
        const int b = l & 1;
        if (l >= 2 && !mbar_wait(&tme[b], ((l - 2) >> 1) & 1, abort)) break;
        tc_after();
        const uint32_t d = tmem + (uint32_t)(b * kMaxCols);
        const uint32_t id = idesc_tf32(ncols);
        bool ok = true;
        for (int kc = 0; kc < Kc; ++kc, ++it) {
          const int s = it % kStages;
          const uint32_t ph = (it / kStages) & 1;
          if (!mbar_wait(&fullA[s], ph, abort) || !mbar_wait(&fullB[s], ph, abort)) { ok = false; break; }
          tc_after();
          const uint32_t a0 = su32(sA + (size_t)s * 2 * (Smem::kA / 4));
          const uint32_t b0 = su32(sB + (size_t)s * 2 * (Smem::kB / 4));
          const uint64_t ahi = sdesc(a0), alo = sdesc(a0 + (uint32_t)Smem::kA);
          const uint64_t bhi = sdesc(b0), blo = sdesc(b0 + (uint32_t)Smem::kB);
          mma_tf32(d, ahi, bhi, id, kc > 0 ? 1u : 0u);
          mma_tf32(d, ahi, blo, id, 1u);
          mma_tf32(d, alo, bhi, id, 1u);
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        mma_commit(&tmf[b]);
      }
      mma_commit(done);
      mbar_drain(done, 0);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int r = tid & (kRows - 1), grp = tid >> 7;   // grp = warp / 4
    const bool valid = rowYZ[2 * r] >= 0;
    const int Y = valid ? rowYZ[2 * r] : 0, Z = valid ? rowYZ[2 * r + 1] : 0;  // safe addresses
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    float* acc = st9 + (size_t)r * PPQ_NA2;
    for (int l = 0; l < nloc; ++l) {
      const int16_t* h = chunks + (size_t)(cb + l) * kChunkFields;
      const int ng = h[2];
      const int b = l & 1;
      // bounded wait; the whole warp agrees before the collective TMEM loads
      bool ok = mbar_wait(&tmf[b], (l >> 1) & 1, abort);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_after();
      for (int j = 0; j < ng; ++j) {
        const int q = h[8 + j];
        const uint32_t col = tmem + lane_base + (uint32_t)(b * kMaxCols + j * Npad);
        for (int ch = ppq_c9qp[q]; ch < ppq_c9qp[q + 1]; ++ch) {
          const int16_t* c = ppq_c9q + 4 * ch;
          if ((c[2] & 3) != grp) continue;                    // warp-uniform
          const float* py = clT + (size_t)c[0] * NNp + Y;     // Cl[W,Y][c3] at W * N
          const float* pz = clT + (size_t)c[1] * NNp + Z;     // Cl[W,Z][c4] at W * N
          float v0 = 0.f, v1 = 0.f;
          // software pipeline: the Cl factors of block W0 + 8 are loaded while
          // the TMEM columns of block W0 are in flight
          float a[8], bz[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            a[i] = i < N ? __ldg(py + i * N) : 0.f;
            bz[i] = i < N ? __ldg(pz + i * N) : 0.f;
          }
#pragma unroll
          for (int W0 = 0; W0 < NW; W0 += 8) {
            uint32_t D[8];
            tmem_issue8(col + (uint32_t)W0, D);
            float an[8], bn[8];
            if (W0 + 8 < NW) {
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const bool in = W0 + 8 + i < N;
                an[i] = in ? __ldg(py + (W0 + 8 + i) * N) : 0.f;
                bn[i] = in ? __ldg(pz + (W0 + 8 + i) * N) : 0.f;
              }
            }
            tmem_wait8(D);
#pragma unroll
            for (int i = 0; i < 8; i += 2) {
              v0 = fmaf(__uint_as_float(D[i]) * a[i], bz[i], v0);
              v1 = fmaf(__uint_as_float(D[i + 1]) * a[i + 1], bz[i + 1], v1);
            }
            if (W0 + 8 < NW) {
#pragma unroll
              for (int i = 0; i < 8; ++i) { a[i] = an[i]; bz[i] = bn[i]; }
            }
          }
          if (valid) acc[c[2]] += 0.5f * float(c[3]) * (v0 + v1);
        }
      }
      tc_before();
      mbar_arrive(&tme[b]);
    }
  }
  tc_before();
  __syncthreads();
  if (tid < kRows) {
    // this CTA's row sums to its slot
    const int p = tile * kRows + tid;
    if (p < P) {
      float* dst = part + ((size_t)(blockIdx.x % nslot) * P + p) * PPQ_NA2;
      for (int o = 0; o < PPQ_NA2; ++o) dst[o] = st9[tid * PPQ_NA2 + o];
    }
  }
  __syncthreads();
  if (*abort && tid == 0) {
    atomicExch(err, 1);
    part[((size_t)(blockIdx.x % nslot) * P + (size_t)tile * kRows) * PPQ_NA2] = __int_as_float(0x7fc00000);  // NaN
  }
  if (warp == kMmaWarp) {
    tc_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kMaxCols)
                 : "memory");
  }
}

}  // namespace tc
}  // namespace ppq
