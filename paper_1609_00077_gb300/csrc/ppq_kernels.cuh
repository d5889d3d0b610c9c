// ppq_kernels.cuh -- CUDA kernels of the PQ residual, energy and update.
//
// The residual R(T) of the PQ model (Theory section: the block decomposition
// of Eq. decompose inserted into the projected CC equations, exact, two-label
// integrals, full Fock matrix) is evaluated in a site formulation: every pair
// label P is a site with a 16-state local Fock space, T and H are written as
// graded products of per-site monomials, and the linked residual
// <mu| exp(-T) H exp(T) |Phi> is summed over the Hamiltonian pieces H_S
// (one- or two-site S).  For each piece only clusters touching S contribute;
// internal clusters are absorbed into the closure Ht_S = exp(-I_S) H_S exp(I_S)
// and the clusters linking S to the output sites enter through the link
// coefficients Cl[X,Y] = components of exp(T_XY)|ref>.  Nine topologies
// (output sites inside or outside S, zero to two summed sites) give the
// residual; the quartic one (two summed sites) is the paper's O(N^4)
// three-label-intermediate class (Table V, kernels o(x,y,z) <- sum_w ...).
// All coefficient tables come from tables.py (ppq_tables.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "ppq_tables.h"

namespace ppq {

__device__ __forceinline__ int unpack_t(int32_t e) { return e >> 17; }
__device__ __forceinline__ int unpack_s(int32_t e) { return (e >> 1) & 0xFFFF; }
template <typename R>
__device__ __forceinline__ R unpack_sign(int32_t e) { return (e & 1) ? R(-1) : R(1); }

// ---------------------------------------------------------------- a1: staging
// f_pq = h_pq + sum_i [2 (pq|ii) - (pi|iq)];  h'_pq keeps the mean field of the
// occupied orbitals whose label lies outside {L(p), L(q)} (those integrals are
// three-label ones, dropped by the two-label truncation).
// two-electron integrals (pq|rs): the dense n^4 array, or a three-index
// factorisation (pq|rs) = sum_Q B[pq][Q] B[rs][Q] (Cholesky vectors; the
// paper builds its integral blocks from such B matrices, Implementation section)
struct EriSrc {
  const double* eri;  // dense, row-major (pq|rs); nullptr for the factorised form
  const double* Bt;   // [n * n][naux]
  int naux;
  int n;
  __device__ __forceinline__ double operator()(int p, int q, int r, int s) const {
    if (eri) {
      size_t n1 = n;
      return eri[((p * n1 + q) * n1 + r) * n1 + s];
    }
    const double* a = Bt + ((size_t)p * n + q) * naux;
    const double* b = Bt + ((size_t)r * n + s) * naux;
    double v = 0.0;
    for (int Q = 0; Q < naux; ++Q) v += a[Q] * b[Q];
    return v;
  }
};

__global__ void k_fock(int n, int N, const double* __restrict__ h, EriSrc E,
                       const int* __restrict__ occ, const int* __restrict__ lab,
                       double* __restrict__ f, double* __restrict__ hp) {
  int pq = blockIdx.x * blockDim.x + threadIdx.x;
  if (pq >= n * n) return;
  int p = pq / n, q = pq % n;
  double mf = 0.0, mfl = 0.0;
  int lp = lab[p], lq = lab[q];
  for (int k = 0; k < N; ++k) {
    int i = occ[k];
    double v = 2.0 * E(p, q, i, i) - E(p, i, i, q);
    mf += v;
    if (k == lp || k == lq) mfl += v;
  }
  f[pq] = h[pq] + mf;
  hp[pq] = (lp == lq) ? h[pq] : h[pq] + mf - mfl;
}

// gather the per-site (20) and per-ordered-pair (232) integrals
template <typename R>
__global__ void k_gather(int n, int N, const double* __restrict__ hp, EriSrc E,
                         const int* __restrict__ occ, const int* __restrict__ vir,
                         R* __restrict__ g1, R* __restrict__ g2) {
  size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t n1 = n;
  size_t tot2 = (size_t)N * N * PPQ_NG2;
  if (tid < tot2) {
    int j = tid % PPQ_NG2;
    int XW = tid / PPQ_NG2;
    int X = XW / N, W = XW % N;
    if (X == W) { g2[tid] = R(0); return; }
    const int8_t* k = ppq_g2key + 5 * j;
    int o[4] = {occ[X], vir[X], occ[W], vir[W]};
    double v;
    if (k[0] == 0) v = hp[o[k[1]] * n1 + o[k[2]]];
    else v = E(o[k[1]], o[k[2]], o[k[3]], o[k[4]]);
    g2[tid] = R(v);
    return;
  }
  tid -= tot2;
  if (tid < (size_t)N * PPQ_NG1) {
    int j = tid % PPQ_NG1, X = tid / PPQ_NG1;
    const int8_t* k = ppq_g1key + 5 * j;
    int o[2] = {occ[X], vir[X]};
    double v;
    if (k[0] == 0) v = hp[o[k[1]] * n1 + o[k[2]]];
    else v = E(o[k[1]], o[k[2]], o[k[3]], o[k[4]]);
    g1[tid] = R(v);
  }
}

// ---------------------------------------------------------------- links
// Cl[X,Y][c] = <c| exp(T_XY) |ref> on the 36-state zero-charge sector
// (c = 0..29 nonzero), exp(T_XY) = prod_k (1 + t_k O_k).
template <typename R>
__global__ void k_links(int N, const double* __restrict__ t2, R* __restrict__ cl) {
  int XY = blockIdx.x * blockDim.x + threadIdx.x;
  if (XY >= N * N) return;
  int X = XY / N, Y = XY % N;
  R v[PPQ_NS36];
#pragma unroll
  for (int c = 0; c < PPQ_NS36; ++c) v[c] = R(0);
  if (X != Y) {
    // generated straight-line operator sequence (ppq_link_apply): constant
    // indices keep v in registers
    v[0] = R(1);
    ppq_link_apply(t2 + (size_t)XY * PPQ_NA2, v);
  }
  R* o = cl + (size_t)XY * PPQ_NS36;
#pragma unroll
  for (int c = 0; c < PPQ_NS36; ++c) o[c] = v[c];
}

// ---------------------------------------------------------------- closures
// one-site closure Ht_X = exp(-T_X) H_X exp(T_X), full 16x16
template <typename R>
__global__ void k_site_closure(int N, const R* __restrict__ g1, const double* __restrict__ t1,
                               R* __restrict__ hs, double* __restrict__ esite) {
  __shared__ R M[256];
  __shared__ R h00;
  int X = blockIdx.x;
  for (int i = threadIdx.x; i < 256; i += blockDim.x) M[i] = R(0);
  __syncthreads();
  const R* g = g1 + (size_t)X * PPQ_NG1;
  for (int el = threadIdx.x; el < PPQ_H1_NEL; el += blockDim.x) {
    R s = R(0);
    for (int p = ppq_h1_ptr[el]; p < ppq_h1_ptr[el + 1]; ++p) s += R(ppq_h1_c[p]) * g[ppq_h1_j[p]];
    M[ppq_h1_el[el]] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) h00 = M[0];
  for (int k = 0; k < 3; ++k) {
    R tk = R(t1[X * 3 + k]);
    for (int e = ppq_s_rptr[k] + threadIdx.x; e < ppq_s_rptr[k + 1]; e += blockDim.x) {
      int32_t w = ppq_s_right[e];
      M[unpack_t(w)] += tk * unpack_sign<R>(w) * M[unpack_s(w)];
    }
    __syncthreads();
  }
  for (int k = 0; k < 3; ++k) {
    R tk = R(t1[X * 3 + k]);
    for (int e = ppq_s_lptr[k] + threadIdx.x; e < ppq_s_lptr[k + 1]; e += blockDim.x) {
      int32_t w = ppq_s_left[e];
      M[unpack_t(w)] -= tk * unpack_sign<R>(w) * M[unpack_s(w)];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < 256; i += blockDim.x) hs[(size_t)X * 256 + i] = M[i];
  if (threadIdx.x == 0) esite[X] = double(M[0]) - double(h00);
}

// two-site closure Ht_XW = exp(-I) H_XW exp(I), I = T_X + T_W + T_XW, on the
// charge/S_z block layout (4900 entries); writes the entries the topologies
// use (G row, T7 entries and their transpose, column 0) and the pair energy.
// Persistent: each CTA stages the output element lists in shared memory once,
// reads the Hamiltonian CSR through L1, and then loops over pairs XW.  Right
// multiplication by (1 + t_o O_o) only mixes entries of one row and left
// multiplication only entries of one column, and every row (column) of a
// sector goes through the same sequence: a thread loads its row into
// registers, runs the sector's generated straight-line sequence of
// multiply-adds over all 35 operators (ppq_sweep_right), stores the row, and
// then does the same for its column (ppq_sweep_left).  Threads are ordered by
// sector, so the lanes of a warp run the same sequence.  The shared copy of M
// pads every sector row to dim + 1 entries (no bank conflicts when the threads
// of a sector load their rows or columns).  The gather multiplies by the five
// coefficient values -1, -1/2, 1/2, 1, 2 through a pre-scaled copy of the
// integrals (the products are exact).  Element for element the arithmetic of
// the flat operator-by-operator sweeps (ppq_p_right / ppq_p_left, used by the
// adjoint's forward recomputation).
struct ClosureSmem {
  static constexpr int kM = PPQ_BLKP + 8;
  static constexpr int kG = PPQ_H2_NCODE * PPQ_NG2 + 8;   // pre-scaled integrals, then zeros
  template <typename R>
  static __host__ __device__ constexpr size_t off_oel() { return ((kM + kG + 72) * sizeof(R) + 15) / 16 * 16; }
  template <typename R>
  static __host__ __device__ constexpr size_t total() {
    return off_oel<R>() + ((PPQ_NS36 + PPQ_NT7E + PPQ_NCOL0) * 2 + 15) / 16 * 16;
  }
};

template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 3 : 2) k_pair_closure_p(int N, const R* __restrict__ g2,
    const double* __restrict__ t1, const double* __restrict__ t2, R* __restrict__ pg,
    R* __restrict__ pt7, R* __restrict__ pc0, double* __restrict__ epair, R* __restrict__ pt7T) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* M = reinterpret_cast<R*>(smem_raw);
  R* gsv = M + ClosureSmem::kM;                          // [code][j]
  R* fac = gsv + ClosureSmem::kG;                        // [2 o + sign], slots 70, 71 = 0
  int16_t* oel = reinterpret_cast<int16_t*>(smem_raw + ClosureSmem::off_oel<R>());
  const int tid = threadIdx.x;
  for (int i = tid; i < PPQ_NS36; i += blockDim.x) oel[i] = ppq_g_elp[i];
  for (int i = tid; i < PPQ_NT7E; i += blockDim.x) oel[PPQ_NS36 + i] = ppq_t7_elp[i];
  for (int i = tid; i < PPQ_NCOL0; i += blockDim.x) oel[PPQ_NS36 + PPQ_NT7E + i] = ppq_col0_elp[i];
  if (tid < 8) gsv[PPQ_H2_NCODE * PPQ_NG2 + tid] = R(0);  // the zero term of the padded streams
  // this thread's row / column (blockDim.x == 256 two-site states, by sector)
  const int st = ppq_th_state[tid];
  const int q = ppq_st_sec[st], dp = ppq_sec_dim[q] + 1;
  const int rowbase = ppq_sec_pbase[q] + ppq_st_pos[st] * dp;
  const int colbase = ppq_sec_pbase[q] + ppq_st_pos[st];
  const int NN = N * N;
  for (int XW = blockIdx.x; XW < NN; XW += gridDim.x) {
    const int X = XW / N, W = XW % N;
    if (X == W) {
      for (int i = tid; i < PPQ_NS36; i += blockDim.x) pg[(size_t)XW * PPQ_NS36 + i] = R(0);
      for (int i = tid; i < PPQ_NT7E; i += blockDim.x) {
        pt7[(size_t)XW * PPQ_NT7E + i] = R(0);
        pt7T[(size_t)i * NN + XW] = R(0);
      }
      for (int i = tid; i < PPQ_NCOL0; i += blockDim.x) pc0[(size_t)XW * PPQ_NCOL0 + i] = R(0);
      if (tid == 0) epair[XW] = 0.0;
      continue;
    }
    if (tid < 36) {
      R to = tid == 35 ? R(0)
                       : R(tid < 3 ? t1[X * 3 + tid] : (tid < 6 ? t1[W * 3 + tid - 3] : t2[(size_t)XW * PPQ_NA2 + tid - 6]));
      fac[2 * tid] = to;
      fac[2 * tid + 1] = -to;
    }
    const R* g = g2 + (size_t)XW * PPQ_NG2;
    for (int i = tid; i < PPQ_NG2; i += blockDim.x) {
      const R v = g[i];
#pragma unroll
      for (int c = 0; c < PPQ_H2_NCODE; ++c) gsv[c * PPQ_NG2 + i] = R(ppq_h2_code[c]) * v;
    }
    for (int i = tid; i < ClosureSmem::kM; i += blockDim.x) M[i] = R(0);
    __syncthreads();
    {
      // the Hamiltonian gather as this thread's term stream (coalesced words
      // read through L1, the same 70 KB for every pair): sum the pre-scaled
      // integrals of an element, store it at its last term
      R acc = R(0);
      const uint32_t* sw = ppq_h2_stream + tid;
#pragma unroll 8
      for (int j = 0; j < PPQ_H2_SLEN; ++j) {
        const uint32_t w = __ldg(sw + (size_t)j * 256);
        acc += gsv[w & 0x7FFu];
        if (w >> 31) {
          M[(w >> 11) & 0x1FFFu] = acc;
          acc = R(0);
        }
      }
    }
    __syncthreads();
    const R h00 = M[PPQ_EL00P];
    // right: M <- M exp(I), this thread's row in registers (generated per sector)
    ppq_sweep_right<R>(q, M, rowbase, fac);
    __syncthreads();
    // left: M <- exp(-I) M, this thread's column in registers
    ppq_sweep_left<R>(q, M, colbase, fac);
    __syncthreads();
    for (int i = tid; i < PPQ_NS36; i += blockDim.x) pg[(size_t)XW * PPQ_NS36 + i] = M[oel[i]];
    for (int i = tid; i < PPQ_NT7E; i += blockDim.x) {
      R v = M[oel[PPQ_NS36 + i]];
      pt7[(size_t)XW * PPQ_NT7E + i] = v;
      pt7T[(size_t)i * NN + (size_t)W * N + X] = v;  // stored [e][W][X]
    }
    for (int i = tid; i < PPQ_NCOL0; i += blockDim.x) pc0[(size_t)XW * PPQ_NCOL0 + i] = M[oel[PPQ_NS36 + PPQ_NT7E + i]];
    if (tid == 0) epair[XW] = double(M[PPQ_EL00P]) - double(h00);
    __syncthreads();
  }
}

// ---------------------------------------------------------------- contractions
template <typename R>
__device__ __forceinline__ R block_sum(R v, R* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  R s = R(0);
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

// r1[Y]: topologies T1 (Ht_Y), T6 (pair pieces on Y,W), T3 (one-site piece on
// X linked to Y), T8 (pair piece on X,W, both linked to Y)
constexpr int kR1Ld = PPQ_NS36 + 1;   // row stride of the staged Cl column in k_r1
template <typename R>
__global__ void k_r1(int N, const R* __restrict__ hs, const R* __restrict__ pc0,
                     const R* __restrict__ cl, const R* __restrict__ gT, double* __restrict__ part) {
  // block (Y, split): the T3 / column-0 part in split 0, the T8 sum over
  // XW = split, split + nsplit, ... ; partial sums to part[split][Y][3].
  // Every link coefficient the block reads is one of Cl[., Y]: the column is
  // staged in shared memory as rows cY[X][c] of kR1Ld (odd) words, so that
  // lanes with consecutive W hit distinct banks; G[X,W][g] comes from the
  // transposed gT[g][X][W] (lanes read consecutive words); the T8 entries
  // are generated straight-line code (ppq_r1_t8), no table reads.
  extern __shared__ __align__(16) unsigned char r1_smem[];
  R* cY = reinterpret_cast<R*>(r1_smem);
  __shared__ R red[32];
  const int Y = blockIdx.x, sp = blockIdx.y, nsp = gridDim.y;
  for (int i = threadIdx.x; i < N * PPQ_NS36; i += blockDim.x) {
    const int X = i / PPQ_NS36, c = i % PPQ_NS36;
    cY[X * kR1Ld + c] = cl[((size_t)X * N + Y) * PPQ_NS36 + c];
  }
  __syncthreads();
  R acc[3] = {R(0), R(0), R(0)};
  for (int X = threadIdx.x; sp == 0 && X < N; X += blockDim.x) {
    if (X == Y) continue;
    const R* h0 = hs + (size_t)X * 256;  // row 0 of Ht_X
    for (int k = 0; k < 3; ++k)
      for (int e = ppq_t3p[k]; e < ppq_t3p[k + 1]; ++e)
        acc[k] += h0[ppq_t3[3 * e + 1]] * cY[X * kR1Ld + ppq_t3[3 * e]];
    const R* p0 = pc0 + ((size_t)Y * N + X) * PPQ_NCOL0;
    for (int k = 0; k < 3; ++k) acc[k] += p0[29 + k];
  }
  const size_t NN = (size_t)N * N;
  for (int XW = sp * blockDim.x + threadIdx.x; XW < N * N; XW += nsp * blockDim.x) {
    int X = XW / N, W = XW % N;
    if (X == W || X == Y || W == Y) continue;
    ppq_r1_t8(cY + X * kR1Ld, cY + W * kR1Ld, gT + XW, NN, acc);
  }
  for (int k = 0; k < 3; ++k) {
    R s = block_sum(acc[k], red);
    if (threadIdx.x == 0) part[((size_t)sp * N + Y) * 3 + k] = double(s);
  }
}

// r1[Y][k] = site element + sum of the k_r1 partial sums in split order
template <typename R>
__global__ void k_r1_reduce(int N, int nsp, const R* __restrict__ hs, const double* __restrict__ part,
                            double* __restrict__ r1) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * N) return;
  int Y = i / 3, k = i % 3;
  double v = 0.0;
  for (int s = 0; s < nsp; ++s) v += part[(size_t)s * 3 * N + i];
  r1[i] = v + double(hs[(size_t)Y * 256 + ppq_A1[k] * 16]);
}

// r2 for ordered (Y,Z): T5, T4 directly (dir) and T2+T7 through the
// exp(-T_YZ) transform (abuf, mirrored later); T9 is the quartic kernels
// (tc::k_t9_tc, tc::k_t9_tc64, k_t9_gemm) and k_t9_reduce
template <typename R>
__global__ void __launch_bounds__(256) k_r2(int N, const R* __restrict__ hs, const R* __restrict__ pc0,
    const R* __restrict__ m7, const R* __restrict__ pg, const R* __restrict__ cl,
    const double* __restrict__ t2, double* __restrict__ dir, double* __restrict__ abuf) {
  __shared__ R U[PPQ_NS36];
  __shared__ R outs[PPQ_NA2];
  int YZ = blockIdx.x;
  int Y = YZ / N, Z = YZ % N;
  if (Y == Z) {
    for (int k = threadIdx.x; k < PPQ_NA2; k += blockDim.x) {
      dir[(size_t)YZ * PPQ_NA2 + k] = 0.0;
      abuf[(size_t)YZ * PPQ_NA2 + k] = 0.0;
    }
    return;
  }
  const R* clYZ = cl + (size_t)YZ * PPQ_NS36;
  constexpr int S7 = 7;
  __shared__ R part7[PPQ_NS36][S7];
  // T4 (direct term, needed for Y < Z only): the rows Cl[X,Y][.], Cl[X,Z][.]
  // and Ht_X[0, 5 / 10 / 15] of every X are staged in shared memory (rows of
  // kR1Ld words, lanes on consecutive X hit distinct banks); thread (X, half)
  // runs the generated entries of outputs 0-14 or 15-28 (a warp per half
  // and 32 X), and the per-X sums go to p4[o][X] (over the staged rows) for
  // a fixed-order sum over X
  extern __shared__ __align__(16) unsigned char r2_smem[];
  R* cY = reinterpret_cast<R*>(r2_smem);          // [N][kR1Ld]
  R* cZ = cY + (size_t)N * kR1Ld;                  // [N][kR1Ld]
  R* hx = cZ + (size_t)N * kR1Ld;                  // [N][3]
  R* p4 = cY;                                      // [29][N], after the T4 sums
  if (Y < Z) {
    for (int i = threadIdx.x; i < N * PPQ_NS36; i += blockDim.x) {
      const int X = i / PPQ_NS36, c = i % PPQ_NS36;
      cY[X * kR1Ld + c] = cl[((size_t)X * N + Y) * PPQ_NS36 + c];
      cZ[X * kR1Ld + c] = cl[((size_t)X * N + Z) * PPQ_NS36 + c];
    }
    for (int i = threadIdx.x; i < 3 * N; i += blockDim.x) hx[i] = hs[(size_t)(i / 3) * 256 + 5 * (i % 3 + 1)];
  }
  __syncthreads();
  const int X4 = ((threadIdx.x >> 6) << 5) | (threadIdx.x & 31), h4 = (threadIdx.x >> 5) & 1;
  const bool do4 = Y < Z && X4 < N;
  static_assert(PPQ_NA2 == 29, "two halves of at most 15 outputs");
  R a4[15];
#pragma unroll
  for (int i = 0; i < 15; ++i) a4[i] = R(0);
  if (do4 && X4 != Y && X4 != Z) {
    if (h4 == 0) ppq_r2_t4_0(cY + X4 * kR1Ld, cZ + X4 * kR1Ld, hx + 3 * X4, a4);
    else ppq_r2_t4_1(cY + X4 * kR1Ld, cZ + X4 * kR1Ld, hx + 3 * X4, a4);
  }
  // T7 from the GEMM products M7[Y,Z][k] = sum_W pt7[Y,W][e] Cl[W,Z][c2]
  // (W = Y and W = Z contribute zero: Cl[Z,Z] = 0, pt7[Y,Y] = 0)
  const R* m7y = m7 + (size_t)YZ * PPQ_NK7;
  if (threadIdx.x < PPQ_NS36 * S7) {
    int nu = threadIdx.x / S7, sl = threadIdx.x % S7;
    R acc = R(0);
    for (int e = ppq_t7p[nu] + sl; e < ppq_t7p[nu + 1]; e += S7) {
      const int16_t* q = ppq_t7g + 4 * e;
      acc += R(q[3]) * clYZ[q[0]] * m7y[q[1]];
    }
    part7[nu][sl] = acc;
  }
  __syncthreads();   // the staged rows are read; p4 reuses them
  if (do4) {
    const int o0 = 15 * h4, no = h4 ? PPQ_NA2 - 15 : 15;
#pragma unroll
    for (int i = 0; i < 15; ++i)
      if (i < no) p4[(o0 + i) * N + X4] = a4[i];
  }
  __syncthreads();
  // outputs: warp w sums outputs o = w, w + 8, ... over X (lane X = ln, ln + 32, ..., then a shuffle tree)
  {
    const int wp = threadIdx.x >> 5, ln = threadIdx.x & 31;
    for (int o = wp; o < PPQ_NA2; o += blockDim.x >> 5) {
      R acc = R(0);
      if (Y < Z) {
        for (int X = ln; X < N; X += 32) acc += p4[o * N + X];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
        acc += pc0[(size_t)YZ * PPQ_NCOL0 + o];
      }
      if (ln == 0) outs[o] = acc;
    }
  }
  if (threadIdx.x >= 64 && threadIdx.x < 64 + PPQ_NS36) {
    int nu = threadIdx.x - 64;
    R acc = R(0);
    const R* hY = hs + (size_t)Y * 256;
    for (int e = ppq_t2p[nu]; e < ppq_t2p[nu + 1]; ++e) {
      const int16_t* q = ppq_t2 + 4 * e;
      acc += clYZ[q[0]] * hY[q[1] * 16 + q[2]];
    }
    for (int sl = 0; sl < S7; ++sl) acc += part7[nu][sl];
    U[nu] = acc;
  }
  __syncthreads();
  // exp(-T_YZ) on U by one thread, as generated straight-line code over
  // registers (ppq_link_unapply), then the transformed elements to abuf
  if (threadIdx.x == 0) {
    R u[PPQ_NS36];
#pragma unroll
    for (int c = 0; c < PPQ_NS36; ++c) u[c] = U[c];
    ppq_link_unapply(t2 + (size_t)YZ * PPQ_NA2, u);
#pragma unroll
    for (int k = 0; k < PPQ_NA2; ++k) abuf[(size_t)YZ * PPQ_NA2 + k] = double(u[1 + k]);
  }
  for (int k = threadIdx.x; k < PPQ_NA2; k += blockDim.x) dir[(size_t)YZ * PPQ_NA2 + k] = double(outs[k]);
}

// r2[Y,Z] = dir[Y,Z] + abuf[Y,Z] + mirror(abuf[Z,Y]).  Both stored
// orientations of a pair get the average of the two evaluations, so the two
// copies of every amplitude stay exactly consistent under the update.
__global__ void k_assemble(int N, const double* __restrict__ dir, const double* __restrict__ abuf,
                           const double* __restrict__ t9, double* __restrict__ r2) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)N * N * PPQ_NA2) return;
  int k = i % PPQ_NA2;
  int YZ = i / PPQ_NA2;
  int Y = YZ / N, Z = YZ % N;
  if (Y == Z) { r2[i] = 0.0; return; }
  if (Y > Z) return;  // written by the (Z,Y) thread's partner below
  int k2 = ppq_a2_swap[k];
  double sg = double(ppq_a2_swsg[k]);
  size_t j = ((size_t)Z * N + Y) * PPQ_NA2 + k2;
  // direct terms (T4, T5) and the quartic term are evaluated for Y < Z; the
  // two transformed pieces (in-S site Y or Z) add
  double a = dir[i] + t9[i] + abuf[i] + sg * abuf[j];
  r2[i] = a;
  r2[j] = sg * a;
}

// make the two stored copies of every two-pair amplitude consistent (upper
// triangle wins) and zero the diagonal
__global__ void k_symmetrize(int N, double* __restrict__ t2) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)N * N * PPQ_NA2) return;
  int k = i % PPQ_NA2;
  int YZ = i / PPQ_NA2;
  int Y = YZ / N, Z = YZ % N;
  if (Y == Z) { t2[i] = 0.0; return; }
  if (Y > Z) return;
  size_t j = ((size_t)Z * N + Y) * PPQ_NA2 + ppq_a2_swap[k];
  t2[j] = double(ppq_a2_swsg[k]) * t2[i];
}

// ---------------------------------------------------------------- reductions / update
// weight of amplitude i in norms and DIIS dots: 1 for t1, 1/2 for each stored
// copy of a two-pair amplitude (so sums run over unique amplitudes)
__device__ __forceinline__ double amp_weight(size_t i, int N) { return i < (size_t)3 * N ? 1.0 : 0.5; }

__device__ __forceinline__ double denom(size_t i, int N, const double* fo, const double* fv, double shift) {
  double d;
  if (i < (size_t)3 * N) {
    int X = i / 3, m = ppq_A1[i % 3];
    d = ppq_nhole[m] * fo[X] - ppq_npart[m] * fv[X];
  } else {
    size_t j = i - 3 * N;
    int k = j % PPQ_NA2;
    int XY = j / PPQ_NA2;
    int X = XY / N, Y = XY % N;
    int a = ppq_A2[2 * k], b = ppq_A2[2 * k + 1];
    d = ppq_nhole[a] * fo[X] - ppq_npart[a] * fv[X] + ppq_nhole[b] * fo[Y] - ppq_npart[b] * fv[Y];
  }
  return d - shift;
}

// Jacobi step: tn = t + r / D, e = tn - t; written to DIIS slot
__global__ void k_jacobi(size_t L, int N, const double* __restrict__ t, const double* __restrict__ r,
                         const double* __restrict__ fo, const double* __restrict__ fv, double shift,
                         double* __restrict__ tn, double* __restrict__ en) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L) return;
  double d = denom(i, N, fo, fv, shift);
  double e = (d != 0.0) ? r[i] / d : 0.0;
  if (i >= (size_t)3 * N) {
    size_t j = i - 3 * N;
    int XY = j / PPQ_NA2;
    if (XY / N == XY % N) e = 0.0;
  }
  tn[i] = t[i] + e;
  en[i] = e;
}

__global__ void k_extrapolate(size_t L, int m, const double* __restrict__ coef, const int* __restrict__ ok,
                              const double* __restrict__ slots, size_t ld, const int* __restrict__ order,
                              double* __restrict__ t) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L || !*ok) return;
  double s = 0.0;
  for (int k = 0; k < m; ++k) s += coef[k] * slots[order[k] * ld + i];
  t[i] = s;
}

}  // namespace ppq

namespace ppq {

// ---------------------------------------------------------------- quartic term (T9) as GEMMs
// out[Y,Z][o] = 1/2 sum_{X,W} sum_ch s Cl[X,Y][c1] Cl[X,Z][c2] G[X,W][g] Cl[W,Y][c3] Cl[W,Z][c4]
// Stage 1 (this kernel): for each (c2, Y) and each (c1, g) of the channel list
//   B[Y][q][Z][W] = sum_X clT[c2][X][Z] * (clT[c1][X][Y] * gT[g][X][W])
// a GEMM with M = Z, N = W, K = X: rows Z <= Y are skipped (Y < Z symmetry).
// Thread (tz, tw) of a 16x16 grid owns rows tz + 16 i and columns tw + 16 j.
template <typename R, int MT>
__global__ void __launch_bounds__(256) k_t9_gemm(int N, int T, int ldc, const R* __restrict__ clT,
    const R* __restrict__ gT, const int* __restrict__ work, double* __restrict__ part) {
  extern __shared__ unsigned char smem_raw[];
  constexpr int KC = 16;
  const int NPD = T * MT;                       // padded row length (zeros beyond N)
  R* As = reinterpret_cast<R*>(smem_raw);      // [KC][NPD]
  R* Bs = As + KC * NPD;                        // [KC][NPD]
  R* Cs = Bs + KC * NPD;                        // [NPD][NPD]  C tile for the epilogue
  // [N][29] per-row sums of this work item, 16-byte aligned after the tiles
  double* acc = reinterpret_cast<double*>(smem_raw + ((2 * KC * NPD + NPD * NPD) * sizeof(R) + 15) / 16 * 16);
  int c2 = work[3 * blockIdx.x], q0 = work[3 * blockIdx.x + 1], q1 = work[3 * blockIdx.x + 2];
  int Y = blockIdx.y;
  int tz = threadIdx.x / T, tw = threadIdx.x % T;
  bool active = tz < T;
  size_t NN = (size_t)N * N;
  const R* a_src = clT + (size_t)c2 * ldc;     // [X][Z]
  int i0 = (Y + 1) / T;                        // first micro-row that can hold Z > Y
  int nth = blockDim.x;
  for (int e = threadIdx.x; e < N * PPQ_NA2; e += nth) acc[e] = 0.0;
  for (int qq = q0; qq < q1; ++qq) {
    int c1 = ppq_q9c[3 * qq], g = ppq_q9c[3 * qq + 1], q = ppq_q9c[3 * qq + 2];
    const R* ys = clT + (size_t)c1 * ldc;      // [X][Y]
    const R* gs = gT + (size_t)g * NN;         // [X][W]
    R accm[MT][MT];
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
      for (int j = 0; j < MT; ++j) accm[i][j] = R(0);
    for (int k0 = 0; k0 < N; k0 += KC) {
      int kc = min(KC, N - k0);
      __syncthreads();
      for (int e = threadIdx.x; e < kc * NPD; e += nth) {
        int kk = e / NPD, z = e - kk * NPD, X = k0 + kk;
        R av = R(0), bv = R(0);
        if (z < N) {
          av = a_src[(size_t)X * N + z];
          bv = ys[(size_t)X * N + Y] * gs[(size_t)X * N + z];
        }
        As[e] = av;
        Bs[e] = bv;
      }
      __syncthreads();
      if (active) {
        const R* ap = As + tz;
        const R* bp = Bs + tw;
        for (int kk = 0; kk < kc; ++kk) {
          R a[MT], b[MT];
#pragma unroll
          for (int i = 0; i < MT; ++i) a[i] = ap[T * i];
#pragma unroll
          for (int j = 0; j < MT; ++j) b[j] = bp[T * j];
#pragma unroll
          for (int i = 0; i < MT; ++i) {
            if (i < i0) continue;
#pragma unroll
            for (int j = 0; j < MT; ++j) accm[i][j] = fma(a[i], b[j], accm[i][j]);
          }
          ap += NPD;
          bp += NPD;
        }
      }
    }
    // fused epilogue: C tile to shared memory, then
    // acc[Z][o] += 1/2 sum_W sum_{ch of q -> o} s C[Z][W] Cl[W,Y][c3] Cl[W,Z][c4];
    // one thread per (output group, Z), so every sum has a fixed order
    if (active) {
#pragma unroll
      for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < MT; ++j) Cs[(tz + T * i) * NPD + tw + T * j] = accm[i][j];
    }
    __syncthreads();
    int g0 = ppq_c9gp[q], ngr = ppq_c9gp[q + 1] - g0;
    int nz = N - (Y + 1);
    for (int e = threadIdx.x; e < ngr * nz; e += nth) {
      int gi = e / nz, Z = Y + 1 + (e - gi * nz);
      const R* crow = Cs + Z * NPD;
      double sum = 0.0;
      int o = 0;
      for (int ch = ppq_c9g[g0 + gi]; ch < ppq_c9g[g0 + gi + 1]; ++ch) {
        const int16_t* c = ppq_c9q + 4 * ch;
        o = c[2];
        const R* y3 = clT + (size_t)c[0] * ldc + Y;   // Cl[W,Y][c3] = clT[c3][W][Y]
        const R* z4 = clT + (size_t)c[1] * ldc + Z;   // Cl[W,Z][c4] = clT[c4][W][Z]
        R v0 = R(0), v1 = R(0), v2 = R(0), v3 = R(0);
        int W = 0;
        for (; W + 3 < N; W += 4) {
          v0 += crow[W] * __ldg(y3 + (size_t)W * N) * __ldg(z4 + (size_t)W * N);
          v1 += crow[W + 1] * __ldg(y3 + (size_t)(W + 1) * N) * __ldg(z4 + (size_t)(W + 1) * N);
          v2 += crow[W + 2] * __ldg(y3 + (size_t)(W + 2) * N) * __ldg(z4 + (size_t)(W + 2) * N);
          v3 += crow[W + 3] * __ldg(y3 + (size_t)(W + 3) * N) * __ldg(z4 + (size_t)(W + 3) * N);
        }
        for (; W < N; ++W) v0 += crow[W] * __ldg(y3 + (size_t)W * N) * __ldg(z4 + (size_t)W * N);
        sum += 0.5 * double(c[3]) * double((v0 + v1) + (v2 + v3));
      }
      acc[Z * PPQ_NA2 + o] += sum;
    }
  }
  // this work item's rows Z > Y, all outputs (zeros included), to its slot:
  // part[item][p][o] with p = Y (2N - Y - 1) / 2 + Z - Y - 1
  __syncthreads();
  size_t P = (size_t)N * (N - 1) / 2;
  size_t pY = (size_t)Y * (2 * N - Y - 1) / 2;
  double* dst = part + ((size_t)blockIdx.x * P + pY) * PPQ_NA2;
  int nz = N - (Y + 1);
  for (int e = threadIdx.x; e < nz * PPQ_NA2; e += nth) dst[e] = acc[(Y + 1) * PPQ_NA2 + e];
}

// t9[Y,Z][o] = sum over slots k of part[k][p(Y, Z)][o] in slot order (Y < Z),
// zero for Y >= Z
template <typename P_>
__global__ void k_t9_reduce(int N, int nslot, const P_* __restrict__ part, double* __restrict__ t9) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t NN = (size_t)N * N;
  if (i >= NN * PPQ_NA2) return;
  int o = (int)(i % PPQ_NA2);
  size_t YZ = i / PPQ_NA2;
  int Y = (int)(YZ / N), Z = (int)(YZ % N);
  double v = 0.0;
  if (Y < Z) {
    size_t P = NN > 0 ? (size_t)N * (N - 1) / 2 : 0;
    size_t p = (size_t)Y * (2 * N - Y - 1) / 2 + (Z - Y - 1);
    const P_* src = part + p * PPQ_NA2 + o;
    for (int k = 0; k < nslot; ++k) v += double(src[(size_t)k * P * PPQ_NA2]);
  }
  t9[i] = v;
}

// transposed link coefficients clT[c][X][Y] = Cl[X,Y][c]; slices ldc apart
// (N^2 rounded up to a multiple of 4, so that every slice is 16-byte aligned)
template <typename R>
__global__ void k_transpose_cl(int N, int ldc, const R* __restrict__ cl, R* __restrict__ clT) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t NN = (size_t)N * N;
  if (i >= NN * PPQ_NS36) return;
  int c = i / NN;
  size_t XY = i % NN;
  clT[(size_t)c * ldc + XY] = cl[XY * PPQ_NS36 + c];
}

// transposed closure row gT[g][X][W] = G[X,W][g]
template <typename R>
__global__ void k_transpose_g(int N, const R* __restrict__ pg, R* __restrict__ gT) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t NN = (size_t)N * N;
  if (i >= NN * PPQ_NS36) return;
  int g = i / NN;
  size_t XW = i % NN;
  gT[i] = pg[XW * PPQ_NS36 + g];
}

}  // namespace ppq


namespace ppq {

// T7 GEMMs: M7[Y,Z][k] = sum_W pt7[Y,W][e] * Cl[W,Z][c2] for the distinct
// (c2, e) = k of the T7 channels, one CTA per k; operands pt7T[e][W][Y] and
// clT[c2][W][Z]; thread grid T x T, micro-tile MT x MT
template <typename R, int MT>
__global__ void __launch_bounds__(256) k_t7_gemm(int N, int T, int ldc, const R* __restrict__ pt7T,
                                                 const R* __restrict__ clT, R* __restrict__ m7) {
  extern __shared__ unsigned char smem_raw[];
  constexpr int KC = 16;
  const int NPD = T * MT;
  R* As = reinterpret_cast<R*>(smem_raw);      // [KC][NPD]  A^T chunk: As[w][y] = A[y][w]
  R* Bs = As + KC * NPD;                        // [KC][NPD]  B chunk:   Bs[w][z]
  int k = blockIdx.x;
  int c2 = ppq_k7[2 * k], e = ppq_k7[2 * k + 1];
  size_t NN = (size_t)N * N;
  const R* A = pt7T + (size_t)e * NN;          // [W][Y]
  const R* Bm = clT + (size_t)c2 * ldc;        // [W][Z]
  int tz = threadIdx.x / T, tw = threadIdx.x % T;
  bool active = tz < T;
  R acc[MT][MT];
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int j = 0; j < MT; ++j) acc[i][j] = R(0);
  for (int k0 = 0; k0 < N; k0 += KC) {
    int kc = min(KC, N - k0);
    __syncthreads();
    for (int x = threadIdx.x; x < kc * NPD; x += blockDim.x) {
      int kk = x / NPD, yz = x - kk * NPD, W = k0 + kk;
      As[x] = yz < N ? A[(size_t)W * N + yz] : R(0);
      Bs[x] = yz < N ? Bm[(size_t)W * N + yz] : R(0);
    }
    __syncthreads();
    if (active) {
      const R* ap = As + tz;
      const R* bp = Bs + tw;
      for (int kk = 0; kk < kc; ++kk) {
        R a[MT], b[MT];
#pragma unroll
        for (int i = 0; i < MT; ++i) a[i] = ap[T * i];
#pragma unroll
        for (int j = 0; j < MT; ++j) b[j] = bp[T * j];
#pragma unroll
        for (int i = 0; i < MT; ++i)
#pragma unroll
          for (int j = 0; j < MT; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        ap += NPD;
        bp += NPD;
      }
    }
  }
  if (active) {
#pragma unroll
    for (int i = 0; i < MT; ++i) {
      int Y = tz + T * i;
      if (Y >= N) continue;
#pragma unroll
      for (int j = 0; j < MT; ++j) {
        int Z = tw + T * j;
        if (Z < N) m7[((size_t)Y * N + Z) * PPQ_NK7 + k] = acc[i][j];
      }
    }
  }
}

}  // namespace ppq
