// Quartic (T9) topology of the FP64 residual on the tensor cores: exact
// integer splitting (Ozaki-type) of the FP64 operands into TF32-exact slices.
//
//   D[p][W] = sum_X A[p][X] B_g[W][X],  A[p][X] = Cl[X,Y][c1] Cl[X,Z][c2],
//   B_g[W][X] = G[X,W][g]
//
// Each row p of A is scaled by 2^-e_p (2^e_p >= max_X |A[p][X]|, from frexp)
// and each B_g by 2^-f_g (2^f_g >= max |G[.,.][g]|); the scaled values are rounded to 42
// bits and cut into six 7-bit slices, a_0 signed (|a_0| <= 128), a_1..a_5 in
// [0, 128):  x = sum_i a_i 2^(-7 (i + 1)).  A slice product is at most 2^14 in
// magnitude, a K sum (K <= 80) below 2^20.4, and the sum over the <= 6 slice
// pairs (i, j) with i + j = g below 2^23: every TMEM accumulator S_g is an
// exact integer in FP32.  With the 21 pairs i + j <= 5,
//   D = 2^(e_p + f_g - 49) sum_g S_g 2^(7 (5 - g)),
// combined in int64 (exact); the dropped pairs i + j >= 6 bound the error by
// about 2e-12 of max|A row| max|B_g| per X term.  The slicing works on the
// bit patterns with integer operations (no FP64 arithmetic in the producers
// but the product A[p][X]).  The W contraction with Cl[W,Y][c3] Cl[W,Z][c4]
// runs in double-float arithmetic on the FP32 pipe (about 2^-46 relative per
// term), with the power of two applied once per row and channel in FP64.
//
// The four groups of four epilogue warps split the channels of a chunk's
// (c1, c2, g) by output: all channels of one output go to one group (so the
// group owns that output's row sums), the outputs spread over the groups by
// channel count (ppq_c9grp, generated).
//
// Same pipeline as k_t9_tc (producers, one MMA thread, 16 epilogue warps,
// bounded waits): chunks hold one g each (six accumulator groups of Npad
// columns fill TMEM, so the accumulator is single-buffered), the Cl slices are
// FP64 and reloaded only when (c1, c2) changes, and the producers hand each
// row's exponent to the epilogue through mbarriers on four buffers (a producer
// runs at most three chunks ahead of the epilogue: two stages ahead of the
// MMAs, which wait for the epilogue of the previous chunk).
#pragma once
#include <cstdint>

namespace ppq {
namespace tc {

constexpr int kSl = 6;            // slices per operand
constexpr int kSlBits = 7;        // bits per slice
constexpr int kStages64 = 2;
static_assert(kSl == 6 && kSlBits == 7, "split6 cuts 42 bits into six 7-bit slices");

// v 2^(42 - e) (|v| < 2^e) rounded to the nearest integer x (ties away from
// zero), by integer operations on the bit pattern of v, then cut into 7-bit
// slices x = sum_i a_i 2^(7 (5 - i)): a_0 signed (|a_0| <= 128), a_1..a_5 in
// [0, 128).  The slices are small integers, converted to FP32 exactly by the
// 1.5 2^23 magic number; no FP64 arithmetic or 64-bit conversion is involved.
__device__ __forceinline__ float small_int_to_float(int a) {   // |a| < 2^22
  return __fsub_rn(__int_as_float(0x4B400000 + a), 12582912.f);
}

__device__ __forceinline__ void split6(double v, int e, float* s) {
  const long long b = __double_as_longlong(v);
  const int ev = (int)((b >> 52) & 0x7FF);
  const long long m = (b & 0x000FFFFFFFFFFFFFLL) | 0x0010000000000000LL;
  // v = m 2^(ev - 1075), so x = round(m 2^-sh) with sh >= 11 for |v| < 2^e
  const int sh = 1075 - kSl * kSlBits + e - ev;
  long long x = 0;
  if (ev != 0 && sh > 0 && sh < 64) x = (m + (1LL << (sh - 1))) >> sh;
  if (b < 0) x = -x;
  const int a0 = (int)(x >> 35);
  const long long r = x - ((long long)a0 << 35);       // [0, 2^35)
  const int rh = (int)(r >> 14), rl = (int)(r & 0x3FFF);
  s[0] = small_int_to_float(a0);
  s[1] = small_int_to_float(rh >> 14);
  s[2] = small_int_to_float((rh >> 7) & 127);
  s[3] = small_int_to_float(rh & 127);
  s[4] = small_int_to_float(rl >> 7);
  s[5] = small_int_to_float(rl & 127);
}

// an exact integer |d| < 2^58 as a float pair d = dh + dl (to 2^-48 |d|):
// limbs d = d2 2^46 + d1 2^23 + d0 (each exact in FP32 through the 2^23
// magic-number conversion), then two fast two-sums, valid because each
// partial sum is zero or at least the next limb in magnitude
__device__ __forceinline__ void dpair(long long d, float& dh, float& dl) {
  const int d2 = (int)(d >> 46);
  const int d1 = (int)((d >> 23) & 0x7FFFFF), d0 = (int)(d & 0x7FFFFF);
  const float f2 = __fmul_rn(__fsub_rn(__int_as_float(0x4B400000 + d2), 12582912.f), 70368744177664.f);
  const float f1 = __fmul_rn(__fsub_rn(__int_as_float(0x4B000000 | d1), 8388608.f), 8388608.f);
  const float f0 = __fsub_rn(__int_as_float(0x4B000000 | d0), 8388608.f);
  const float x = __fadd_rn(f2, f1), e1 = __fsub_rn(f1, __fsub_rn(x, f2));
  dh = __fadd_rn(x, f0);
  const float e2 = __fsub_rn(f0, __fsub_rn(dh, x));
  dl = __fadd_rn(e1, e2);
}

// the link coefficients of the epilogue as float pairs: clT2[i] = (hi, lo),
// hi = x rounded to FP32, lo = (x - hi) rounded (hi + lo = x to 2^-48)
__global__ void k_split_cl(size_t n, const double* __restrict__ clT, float2* __restrict__ clT2) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = clT[i];
  const float hi = __double2float_rn(x);
  clT2[i] = make_float2(hi, __double2float_rn(x - (double)hi));
}

// B slices per K stage: bpre64[g][j][kc][W / 8][kcore][W % 8][k % 4] (value
// slice j of G[X,W][g] 2^-f_g), X = 8 kc + 4 kcore + k % 4; one block per g,
// the exponent f_g (0 for an all-zero g) in fexp[g]
__global__ void __launch_bounds__(128) k_t9_bprep64(int N, int Npad, int Kc, const double* __restrict__ pg,
                                                    float* __restrict__ bpre, int* __restrict__ fexp) {
  __shared__ double red[128];
  const int g = blockIdx.x, tid = threadIdx.x;
  double mx = 0.0;
  for (int i = tid; i < N * N; i += blockDim.x) mx = fmax(mx, fabs(pg[(size_t)i * PPQ_NS36 + g]));
  red[tid] = mx;
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (tid < o) red[tid] = fmax(red[tid], red[tid + o]);
    __syncthreads();
  }
  int f = 0;
  if (red[0] > 0.0) frexp(red[0], &f);
  if (tid == 0) fexp[g] = f;
  const size_t per = (size_t)Npad * 8;
  for (int i = tid; i < Kc * 8 * Npad; i += blockDim.x) {
    const int X = i / Npad, W = i % Npad;
    const double v = (W < N && X < N) ? pg[((size_t)X * N + W) * PPQ_NS36 + g] : 0.0;
    float sl[kSl];
    split6(v, f, sl);
    const int kc = X >> 3, k = X & 7, kcore = k >> 2, e = k & 3;
    const size_t off = ((size_t)((W >> 3) * 2 + kcore) * 8 + (W & 7)) * 4 + e;
#pragma unroll
    for (int j = 0; j < kSl; ++j) bpre[((size_t)(g * kSl + j) * Kc + kc) * per + off] = sl[j];
  }
}

struct Smem64 {
  static constexpr size_t kA = (size_t)kRows * 8 * 4;           // one slice of one A stage
  static constexpr size_t kB = (size_t)96 * 8 * 4;              // one slice of one B stage (Npad <= 96)
  static constexpr size_t kStageBytes = kSl * (kA + kB);
  static constexpr int kNBars = 3 * kStages64 + 10;
  static size_t __host__ __device__ slices() { return (size_t)kStages64 * kStageBytes; }
  static size_t __host__ __device__ t9(int NNp) { return slices() + 2 * (size_t)NNp * 8; }
  static size_t __host__ __device__ rows(int NNp) { return t9(NNp) + (size_t)kRows * PPQ_NA2 * 8; }
  static size_t __host__ __device__ bars(int NNp) { return rows(NNp) + (size_t)kRows * 6 * 4; }
  static size_t __host__ __device__ total(int NNp) { return bars(NNp) + kNBars * 8 + 16; }
};

// chunk records as for k_t9_tc, one g per chunk (n_cols = Npad)
template <int NW>
__global__ void __launch_bounds__(kThreads, 1)
    k_t9_tc64(int N, int P, int Kc, int NNp, const double* __restrict__ clT, const float2* __restrict__ clT2,
              const float* __restrict__ bpre, const int* __restrict__ fexp, const int* __restrict__ cta,
              const int16_t* __restrict__ chunks, int nslot, double* __restrict__ part, int* __restrict__ err) {
  constexpr int Npad = NW;
  extern __shared__ __align__(1024) unsigned char sm[];
  float* sA = reinterpret_cast<float*>(sm);                                     // [S][6][128 x 8]
  float* sB = reinterpret_cast<float*>(sm + kStages64 * kSl * Smem64::kA);      // [S][6][96 x 8]
  double* sCl = reinterpret_cast<double*>(sm + Smem64::slices());               // [2][NNp] (c1, c2)
  double* st9 = reinterpret_cast<double*>(sm + Smem64::t9(NNp));                // [128][29]
  int* rowYZ = reinterpret_cast<int*>(sm + Smem64::rows(NNp));                  // [128][2]
  int* rowE = rowYZ + 2 * kRows;                                                // [4][128]
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + Smem64::bars(NNp));
  uint64_t* fullA = bars;                       // [S] count 256
  uint64_t* fullB = bars + kStages64;           // [S] count 1 + tx
  uint64_t* empty = bars + 2 * kStages64;       // [S] commit
  uint64_t* done = bars + 3 * kStages64;        // commit
  uint64_t* slf = done + 1;                     // Cl slices landed (count 1 + tx)
  uint64_t* sle = slf + 1;                      // producers done with the slices (count 256)
  uint64_t* tmf = sle + 1;                      // accumulators ready (commit)
  uint64_t* tme = tmf + 1;                      // epilogue done with TMEM (count 512)
  uint64_t* ref = tme + 1;                      // [4] row exponents written (count 128)
  uint32_t* tbase = reinterpret_cast<uint32_t*>(bars + Smem64::kNBars);
  volatile int* abort = reinterpret_cast<volatile int*>(tbase + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = cta[3 * blockIdx.x], cb = cta[3 * blockIdx.x + 1], ce = cta[3 * blockIdx.x + 2];
  const int nloc = ce - cb;
  const size_t blk = (size_t)Npad * 8;

  if (tid == 0) {
    for (int s = 0; s < kStages64; ++s) {
      mbar_init(&fullA[s], kProdThreads);
      mbar_init(&fullB[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    mbar_init(slf, 1);
    mbar_init(sle, kProdThreads);
    mbar_init(tmf, 1);
    mbar_init(tme, kEpiThreads);
    for (int b = 0; b < 4; ++b) mbar_init(&ref[b], 128);
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
    for (int o = 0; o < PPQ_NA2; ++o) st9[tid * PPQ_NA2 + o] = 0.0;
  }
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
    int issued_b = 0, fills = 0;   // stage fills / slice fills by the lead thread
    int it = 0, e = 0;
    int16_t c1 = -1, c2 = -1;
    for (int l = 0; l < nloc && !*abort; ++l) {
      const int16_t* h = chunks + (size_t)(cb + l) * kChunkFields;
      if (h[0] != c1 || h[1] != c2) {
        // new link pair: reload the FP64 slices once every producer is done
        // with the old ones, then this row's exponent
        if (fills > 0) {
          mbar_arrive(sle);
          if (!mbar_wait(sle, (fills - 1) & 1, abort)) break;
        }
        if (lead) {
          mbar_arrive_tx(slf, 2u * NNp * 8);
          bulk_g2s(sCl, clT + (size_t)h[0] * NNp, NNp * 8, slf);
          bulk_g2s(sCl + NNp, clT + (size_t)h[1] * NNp, NNp * 8, slf);
        }
        ++fills;
        if (!mbar_wait(slf, (fills - 1) & 1, abort)) break;
        c1 = h[0];
        c2 = h[1];
        double mx = 0.0;
        if (Y >= 0)
          for (int X = 0; X < N; ++X) mx = fmax(mx, fabs(sCl[X * N + Y] * sCl[NNp + X * N + Z]));
        e = 0;
        if (mx > 0.0) frexp(mx, &e);
      }
      if (hh == 0) {   // both threads of a row found the same exponent
        rowE[(l & 3) * kRows + r] = e;
        mbar_arrive(&ref[l & 3]);
      }
      const int g = h[4];
      for (int kc = 0; kc < Kc; ++kc, ++it) {
        const int s = it % kStages64;
        const uint32_t ph = (it / kStages64) & 1;
        if (!mbar_wait(&empty[s], ph ^ 1, abort)) break;
        float* bdst = sB + (size_t)s * kSl * (Smem64::kB / 4);
        if (lead) {
          mbar_arrive_tx(&fullB[s], (uint32_t)(kSl * blk * 4));
          for (int j = 0; j < kSl; ++j)
            bulk_g2s(bdst + j * (Smem64::kB / 4), bpre + ((size_t)(g * kSl + j) * Kc + kc) * blk,
                     (uint32_t)(blk * 4), &fullB[s]);
          ++issued_b;
        }
        float sl[4][kSl];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int X = kc * 8 + 4 * hh + k;
          const double a = (Y >= 0 && X < N) ? sCl[X * N + Y] * sCl[NNp + X * N + Z] : 0.0;
          split6(a, e, sl[k]);
        }
        float* adst = sA + (size_t)s * kSl * (Smem64::kA / 4);
        const int base = (r >> 3) * 64 + (r & 7) * 4 + hh * 32;   // this thread's K core
#pragma unroll
        for (int i = 0; i < kSl; ++i)
          *reinterpret_cast<float4*>(adst + i * (Smem64::kA / 4) + base) =
              make_float4(sl[0][i], sl[1][i], sl[2][i], sl[3][i]);
        fence_async_smem();
        mbar_arrive(&fullA[s]);
      }
    }
    if (lead) {
      for (int k = (issued_b > kStages64 ? issued_b - kStages64 : 0); k < issued_b; ++k)
        mbar_drain(&fullB[k % kStages64], (k / kStages64) & 1);
      if (fills > 0) mbar_drain(slf, (fills - 1) & 1);
    }
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      int it = 0;
      const uint32_t id = idesc_tf32(Npad);
      for (int l = 0; l < nloc && !*abort; ++l) {
        if (l >= 1 && !mbar_wait(tme, (l - 1) & 1, abort)) break;
        tc_after();
        bool ok = true;
        for (int kc = 0; kc < Kc; ++kc, ++it) {
          const int s = it % kStages64;
          const uint32_t ph = (it / kStages64) & 1;
          if (!mbar_wait(&fullA[s], ph, abort) || !mbar_wait(&fullB[s], ph, abort)) { ok = false; break; }
          tc_after();
          const uint32_t a0 = su32(sA + (size_t)s * kSl * (Smem64::kA / 4));
          const uint32_t b0 = su32(sB + (size_t)s * kSl * (Smem64::kB / 4));
#pragma unroll
          for (int gg = 0; gg < kSl; ++gg)
#pragma unroll
            for (int i = 0; i <= gg; ++i) {
              const int j = gg - i;
              mma_tf32(tmem + (uint32_t)(gg * Npad), sdesc(a0 + (uint32_t)(i * Smem64::kA)),
                       sdesc(b0 + (uint32_t)(j * Smem64::kB)), id, (kc > 0 || i > 0) ? 1u : 0u);
            }
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        mma_commit(tmf);
      }
      mma_commit(done);
      mbar_drain(done, 0);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int r = tid & (kRows - 1), grp = tid >> 7;
    const bool valid = rowYZ[2 * r] >= 0;
    const int Y = valid ? rowYZ[2 * r] : 0, Z = valid ? rowYZ[2 * r + 1] : 0;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    double* acc = st9 + (size_t)r * PPQ_NA2;
    for (int l = 0; l < nloc; ++l) {
      const int16_t* h = chunks + (size_t)(cb + l) * kChunkFields;
      bool ok = mbar_wait(tmf, l & 1, abort) && mbar_wait(&ref[l & 3], (l >> 2) & 1, abort);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_after();
      const int g = h[4], q = h[8];
      const double rscale = ldexp(1.0, rowE[(l & 3) * kRows + r] + fexp[g] - kSlBits * (kSl + 1));
      for (int ch = ppq_c9qp[q]; ch < ppq_c9qp[q + 1]; ++ch) {
        const int16_t* c = ppq_c9q + 4 * ch;
        if (ppq_c9grp[ch] != grp) continue;                   // warp-uniform; one group per output
        // the W contraction on the FP32 pipe in double-float arithmetic: the
        // link coefficients come as float pairs (hi, lo), so a b = p + pe to
        // 2^-48 (a two-product); the exact integer combination D of the slice
        // accumulators becomes a float pair (dh, dl) through three exact
        // 23-bit limbs and two fast two-sums; the terms D a b accumulate in
        // (vh, vl) with a two-sum
        const float2* py = clT2 + (size_t)c[0] * NNp + Y;
        const float2* pz = clT2 + (size_t)c[1] * NNp + Z;
        float vh = 0.f, vl = 0.f;
#pragma unroll 2
        for (int W0 = 0; W0 < NW; W0 += 4) {
          float2 a[4], b[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const bool in = W0 + i < N;
            a[i] = in ? __ldg(py + (size_t)(W0 + i) * N) : make_float2(0.f, 0.f);
            b[i] = in ? __ldg(pz + (size_t)(W0 + i) * N) : make_float2(0.f, 0.f);
          }
          long long dint[4] = {0, 0, 0, 0};
#pragma unroll
          for (int gg = 0; gg < kSl; ++gg) {
            float sv[4];
            tmem_ld4(tmem + lane_base + (uint32_t)(gg * Npad + W0), sv);
#pragma unroll
            for (int i = 0; i < 4; ++i) dint[i] += (long long)__float2int_rn(sv[i]) << (kSlBits * (kSl - 1 - gg));
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            float dh, dl;
            dpair(dint[i], dh, dl);
            const float p = __fmul_rn(a[i].x, b[i].x);
            float pe = fmaf(a[i].x, b[i].x, -p);
            pe = fmaf(a[i].x, b[i].y, pe);
            pe = fmaf(a[i].y, b[i].x, pe);
            const float hp = __fmul_rn(dh, p);
            float he = fmaf(dh, p, -hp);
            he = fmaf(dh, pe, he);
            he = fmaf(dl, p, he);
            const float sm2 = __fadd_rn(vh, hp), bb = __fsub_rn(sm2, vh);
            vl += __fadd_rn(__fsub_rn(vh, __fsub_rn(sm2, bb)), __fsub_rn(hp, bb)) + he;
            vh = sm2;
          }
        }
        double v = (double)vh + (double)vl;
        v *= rscale;
        if (valid) acc[c[2]] += 0.5 * double(c[3]) * v;
      }
      tc_before();
      mbar_arrive(tme);
    }
  }
  tc_before();
  __syncthreads();
  if (tid < kRows) {
    const int p = tile * kRows + tid;
    if (p < P) {
      double* dst = part + ((size_t)(blockIdx.x % nslot) * P + p) * PPQ_NA2;
      for (int o = 0; o < PPQ_NA2; ++o) dst[o] = st9[tid * PPQ_NA2 + o];
    }
  }
  __syncthreads();
  if (*abort && tid == 0) {
    atomicExch(err, 1);
    part[((size_t)(blockIdx.x % nslot) * P + (size_t)tile * kRows) * PPQ_NA2] =
        __longlong_as_double(0x7ff8000000000000LL);  // NaN
  }
  if (warp == kMmaWarp) {
    tc_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kMaxCols)
                 : "memory");
  }
}

}  // namespace tc
}  // namespace ppq
