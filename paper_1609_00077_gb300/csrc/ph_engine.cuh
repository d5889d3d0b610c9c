// ph_engine.cuh -- the PH (three-pair) residual and solver on the GPU by the
// label-subset expansion; included at the end of ppq_capi.cu (shares its error
// handling and staging helpers).
//
// Exactness (Theory section: amplitudes and integrals block-decomposed by
// pairing labels).  Write the bare Hamiltonian as H = sum_S H_S, H_S the
// integrals (one-body h' and (pq|rs) truncated to <= K_H labels, Table I)
// whose orbitals carry exactly the label set S.  The linked residual of an
// output mu on labels M collects, for each piece S, only amplitudes inside
// U = M + S, so every contribution has a definite label set U with
// |U| <= K + K_H.  The residual of the problem restricted to a label subset L
// (amplitudes and pieces inside L, the same bare pieces) is the sum of the
// contributions with U inside L; Moebius inversion over subsets gives
//     R_mu = sum_{L containing M, |L| <= K + K_H} c_|L| R^(L)_mu,
//     c_k  = sum_{j=0}^{K+K_H-k} (-1)^j C(N - k, j),
// and the energy the same with K_H in place of K + K_H and M empty.
// Each local problem is solved exactly in the site basis of its k <= 6 labels
// (ph_tables.cuh): psi = exp(T)|ref> over the zero-charge sector, phi = <kappa|
// (H - E_0) |psi> on the outputs, R_mu by back-substitution with exp(-T).
#pragma once
#include "ph_tables.cuh"

extern "C" {

/* Host-only export of the structure tables (used by the CPU checks). */
int ph_tables_counts(int k, int K, int K_H, int64_t* counts) {
  int rc;
  const ph::Tables* T = ph::host_tables(k, K, K_H, &rc);
  if (!T) return fail(-1, "ph_tables: cannot build tables for k=%d K=%d K_H=%d (%d)", k, K, K_H, rc);
  const ph::AdjTables* A = ph::host_adjoint(k, K, K_H, &rc);
  if (!A) return fail(-1, "ph_tables: cannot build adjoint tables for k=%d (%d)", k, rc);
  int64_t c[48] = {(int64_t)T->code.size(), (int64_t)T->lvl_ptr.size(), (int64_t)T->ent_ptr.size(),
                   (int64_t)T->ent_sub.size(), (int64_t)T->ent_slot.size(), (int64_t)T->slot_desc.size(),
                   (int64_t)T->out_state.size(), (int64_t)T->out_desc.size(), (int64_t)T->olvl_ptr.size(),
                   (int64_t)T->olvl_order.size(), (int64_t)T->oent_ptr.size(), (int64_t)T->oent_sub.size(),
                   (int64_t)T->oent_slot.size(), (int64_t)T->key_desc.size(), (int64_t)T->h_ptr.size(),
                   (int64_t)T->h_s.size(), (int64_t)T->h_key.size(), (int64_t)T->h_c.size(),
                   (int64_t)T->e0_key.size(), (int64_t)T->e0_c.size(), (int64_t)T->b_ptr.size(),
                   (int64_t)T->b_k.size(), (int64_t)T->b_w.size(), (int64_t)T->d_ptr.size(),
                   (int64_t)T->d_key.size(), (int64_t)T->d_c.size(),
                   (int64_t)A->bs_ptr.size(), (int64_t)A->bs_ent.size(), (int64_t)A->bl_ptr.size(),
                   (int64_t)A->bl_ent.size(), (int64_t)A->obs_ptr.size(), (int64_t)A->obs_ent.size(),
                   (int64_t)A->obl_ptr.size(), (int64_t)A->obl_ent.size(), (int64_t)A->hs_ptr.size(),
                   (int64_t)A->hs_ent.size(), (int64_t)A->hk_ptr.size(), (int64_t)A->hk_ent.size(),
                   (int64_t)A->dk_ptr.size(), (int64_t)A->dk_out.size(), (int64_t)A->dk_c.size(),
                   (int64_t)A->e0_by_key.size(), (int64_t)A->bk_ptr.size(), (int64_t)A->bk_ent.size(),
                   (int64_t)A->bw_ptr.size(), (int64_t)A->bw_ent.size(), (int64_t)A->out_of_state.size(), 0};
  memcpy(counts, c, sizeof c);
  return 0;
}

int ph_tables_copy(int k, int K, int K_H, int which, void* dst) {
  int rc;
  const ph::Tables* T = ph::host_tables(k, K, K_H, &rc);
  if (!T) return fail(-1, "ph_tables: cannot build tables for k=%d K=%d K_H=%d (%d)", k, K, K_H, rc);
  const ph::AdjTables* A = ph::host_adjoint(k, K, K_H, &rc);
  if (!A) return fail(-1, "ph_tables: cannot build adjoint tables for k=%d (%d)", k, rc);
  auto cp = [&](const auto& v) {
    memcpy(dst, v.data(), v.size() * sizeof(v[0]));
    return 0;
  };
  switch (which) {
    case 0: return cp(T->code);
    case 1: return cp(T->lvl_ptr);
    case 2: return cp(T->ent_ptr);
    case 3: return cp(T->ent_sub);
    case 4: return cp(T->ent_slot);
    case 5: return cp(T->slot_desc);
    case 6: return cp(T->out_state);
    case 7: return cp(T->out_desc);
    case 8: return cp(T->olvl_ptr);
    case 9: return cp(T->olvl_order);
    case 10: return cp(T->oent_ptr);
    case 11: return cp(T->oent_sub);
    case 12: return cp(T->oent_slot);
    case 13: return cp(T->key_desc);
    case 14: return cp(T->h_ptr);
    case 15: return cp(T->h_s);
    case 16: return cp(T->h_key);
    case 17: return cp(T->h_c);
    case 18: return cp(T->e0_key);
    case 19: return cp(T->e0_c);
    case 20: return cp(T->b_ptr);
    case 21: return cp(T->b_k);
    case 22: return cp(T->b_w);
    case 23: return cp(T->d_ptr);
    case 24: return cp(T->d_key);
    case 25: return cp(T->d_c);
    case 26: return cp(A->bs_ptr);
    case 27: return cp(A->bs_ent);
    case 28: return cp(A->bl_ptr);
    case 29: return cp(A->bl_ent);
    case 30: return cp(A->obs_ptr);
    case 31: return cp(A->obs_ent);
    case 32: return cp(A->obl_ptr);
    case 33: return cp(A->obl_ent);
    case 34: return cp(A->hs_ptr);
    case 35: return cp(A->hs_ent);
    case 36: return cp(A->hk_ptr);
    case 37: return cp(A->hk_ent);
    case 38: return cp(A->dk_ptr);
    case 39: return cp(A->dk_out);
    case 40: return cp(A->dk_c);
    case 41: return cp(A->e0_by_key);
    case 42: return cp(A->bk_ptr);
    case 43: return cp(A->bk_ent);
    case 44: return cp(A->bw_ptr);
    case 45: return cp(A->bw_ent);
    case 46: return cp(A->out_of_state);
    default: return fail(-2, "ph_tables_copy: unknown table %d", which);
  }
}

}  // extern "C"

namespace ph {

// ------------------------------------------------------------ device constants
__constant__ int8_t c_A3[303 * 3];      // three-pair channel monomials
__constant__ int16_t c_A3inv[4096];     // (a << 8 | b << 4 | c) -> channel, -1 if none
__constant__ int8_t c_key[4][576 * 5];  // integral keys of 1..4 sites: (type, p, q, r, s)
__constant__ int c_binom[128 * 8];      // C(n, r), n < 128, r < 8

constexpr int kNA3 = 303;
constexpr int kNK3 = 576;

__host__ __device__ inline int binom_hd(int n, int r) {
  if (r < 0 || r > n) return 0;
  int c = 1;
  for (int i = 1; i <= r; ++i) c = c * (n - r + i) / i;
  return c;
}

// layout offsets of the K = 3 layout: t1 [N][3], t2 [N][N][29], t3 [N][N][N][303]
__host__ __device__ inline size_t off3(int N) { return (size_t)3 * N + (size_t)29 * N * N; }
inline size_t layout_len(int N, int K) { return K == 3 ? off3(N) + (size_t)kNA3 * N * N * N : off3(N); }

// 1 for the sorted-label ("unique") slots of the layout, 0 for the other stored orders
__device__ __forceinline__ int is_unique(size_t i, int N) {
  if (i < (size_t)3 * N) return 1;
  if (i < off3(N)) {
    size_t q = (i - 3 * N) / 29;
    return (int)(q / N) < (int)(q % N);
  }
  size_t q = (i - off3(N)) / kNA3;
  int R = q % N, Q = (q / N) % N, P = q / ((size_t)N * N);
  return P < Q && Q < R;
}

// excitation rank (number of holes) of the amplitude at layout index i
__device__ __forceinline__ int slot_rank(size_t i, int N) {
  if (i < (size_t)3 * N) return ppq_nhole[ppq_A1[i % 3]];
  if (i < off3(N)) {
    int ch = (i - 3 * N) % 29;
    return ppq_nhole[ppq_A2[2 * ch]] + ppq_nhole[ppq_A2[2 * ch + 1]];
  }
  int ch = (i - off3(N)) % kNA3;
  return ppq_nhole[c_A3[3 * ch]] + ppq_nhole[c_A3[3 * ch + 1]] + ppq_nhole[c_A3[3 * ch + 2]];
}

// a unique slot that the excitation-rank mask keeps (mr = 0: every rank;
// Conclusions: higher excitations disabled)
__device__ __forceinline__ int is_active(size_t i, int N, int mr) {
  return is_unique(i, N) && (mr == 0 || slot_rank(i, N) <= mr);
}

// orbital-energy denominator of a unique slot (Implementation section)
__device__ __forceinline__ double denom3(size_t i, int N, const double* fo, const double* fv, double shift) {
  int lab[3], mon[3], m;
  if (i < (size_t)3 * N) {
    m = 1; lab[0] = i / 3; mon[0] = ppq_A1[i % 3];
  } else if (i < off3(N)) {
    size_t j = i - 3 * N;
    int ch = j % 29; size_t q = j / 29;
    m = 2; lab[0] = q / N; lab[1] = q % N; mon[0] = ppq_A2[2 * ch]; mon[1] = ppq_A2[2 * ch + 1];
  } else {
    size_t j = i - off3(N);
    int ch = j % kNA3; size_t q = j / kNA3;
    m = 3; lab[2] = q % N; lab[1] = (q / N) % N; lab[0] = q / ((size_t)N * N);
    for (int x = 0; x < 3; ++x) mon[x] = c_A3[3 * ch + x];
  }
  double d = 0.0;
  for (int x = 0; x < m; ++x) d += ppq_nhole[mon[x]] * fo[lab[x]] - ppq_npart[mon[x]] * fv[lab[x]];
  return d - shift;
}

// ------------------------------------------------------------ staging
// G1[X][20], G2[X][W][232] (X < W), G3[X][Y][Z][576] (X < Y < Z) and, with
// four-label integrals, G4[rank of X < Y < Z < V][384] from the bare one-body
// part hb and (pq|rs)
constexpr int kNK4 = 384;
__global__ void k_stage_g(int n, int N, int KH, const double* __restrict__ hb, ppq::EriSrc E,
                          const int* __restrict__ occ, const int* __restrict__ vir, const int8_t* __restrict__ subs4,
                          int nsub4, double* __restrict__ G1, double* __restrict__ G2, double* __restrict__ G3,
                          double* __restrict__ G4) {
  size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t n1 = n;
  size_t t1 = (size_t)N * 20, t2 = (size_t)N * N * 232, t3 = KH >= 3 ? (size_t)N * N * N * kNK3 : 0;
  size_t t4 = KH >= 4 ? (size_t)nsub4 * kNK4 : 0;
  int m, j, L[4];
  double* dst;
  if (tid < t1) { m = 1; j = tid % 20; L[0] = tid / 20; dst = G1 + tid; }
  else if ((tid -= t1) < t2) {
    m = 2; j = tid % 232; size_t q = tid / 232; L[0] = q / N; L[1] = q % N; dst = G2 + tid;
    if (L[0] >= L[1]) { *dst = 0.0; return; }
  } else if ((tid -= t2) < t3) {
    m = 3; j = tid % kNK3; size_t q = tid / kNK3; L[2] = q % N; L[1] = (q / N) % N; L[0] = q / ((size_t)N * N);
    dst = G3 + tid;
    if (!(L[0] < L[1] && L[1] < L[2])) { *dst = 0.0; return; }
  } else if ((tid -= t3) < t4) {
    m = 4; j = tid % kNK4; size_t q = tid / kNK4;
    for (int x = 0; x < 4; ++x) L[x] = subs4[q * 4 + x];
    dst = G4 + tid;
  } else return;
  int o[8];
  for (int x = 0; x < m; ++x) { o[2 * x] = occ[L[x]]; o[2 * x + 1] = vir[L[x]]; }
  const int8_t* k = c_key[m - 1] + 5 * j;
  *dst = k[0] == 0 ? hb[o[k[1]] * n1 + o[k[2]]] : E(o[k[1]], o[k[2]], o[k[3]], o[k[4]]);
}

// ------------------------------------------------------------ local problems
// tl[slot][p]: amplitude of cluster slot for the p-th subset of the chunk
template <typename R>
__global__ void k_gather_amp(int P, int p0, int nsub, int k, int nslot, const int* __restrict__ slot_desc,
                             const int8_t* __restrict__ subs, int N, const double* __restrict__ t,
                             R* __restrict__ tl) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)nslot * P) return;
  int slot = i / P, p = i % P;
  R v = R(0);
  if (p0 + p < nsub) {
    int d = slot_desc[slot];
    int m = d & 15, ch = d >> kDescIdx;
    const int8_t* L = subs + (size_t)(p0 + p) * k;
    size_t a = L[(d >> 4) & 15], idx;
    if (m == 1) idx = 3 * a + ch;
    else {
      size_t b = L[(d >> 8) & 15];
      if (m == 2) idx = 3 * (size_t)N + (a * N + b) * 29 + ch;
      else idx = off3(N) + ((a * N + b) * N + (size_t)L[(d >> 12) & 15]) * kNA3 + ch;
    }
    v = R(t[idx]);
  }
  tl[i] = v;
}

// vl[key slot][p]: integral of key slot for the p-th subset
__device__ __forceinline__ int colex_d(const int* p, int m);
template <typename R>
__global__ void k_gather_int(int P, int p0, int nsub, int k, int nkey, const int* __restrict__ key_desc,
                             const int8_t* __restrict__ subs, int N, const double* __restrict__ G1,
                             const double* __restrict__ G2, const double* __restrict__ G3,
                             const double* __restrict__ G4, R* __restrict__ vl) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)nkey * P) return;
  int ks = i / P, p = i % P;
  R v = R(0);
  if (p0 + p < nsub) {
    int d = key_desc[ks];
    int m = d & 15, j = d >> kDescIdx;
    const int8_t* L = subs + (size_t)(p0 + p) * k;
    size_t a = L[(d >> 4) & 15];
    if (m == 1) v = R(G1[a * 20 + j]);
    else {
      size_t b = L[(d >> 8) & 15];
      if (m == 2) v = R(G2[(a * N + b) * 232 + j]);
      else if (m == 3) v = R(G3[((a * N + b) * N + (size_t)L[(d >> 12) & 15]) * kNK3 + j]);
      else {
        int q[4] = {(int)a, (int)b, L[(d >> 12) & 15], L[(d >> 16) & 15]};
        v = R(G4[(size_t)colex_d(q, 4) * kNK4 + j]);
      }
    }
  }
  vl[i] = v;
}

// psi(ref) = psi_minus(ref) = 1, and E_0 = <ref|H|ref> of every subset of the
// chunk (FP64, from the gathered integrals)
template <typename R>
__global__ void k_set_ref(int P, R* __restrict__ a, R* __restrict__ b, int ne0, const int16_t* __restrict__ e0key,
                          const double* __restrict__ e0c, const R* __restrict__ vl, double* __restrict__ e0) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  a[p] = R(1);
  b[p] = R(1);
  double s = 0.0;
  for (int e = 0; e < ne0; ++e) s += e0c[e] * double(vl[(size_t)e0key[e] * P + p]);
  e0[p] = s;
}

// One level of psi = exp(+-T)|ref>: warp per state, lane per J subsets
// (p, p + 32, ...).  Entries i of [s0, s1) (positions in level order);
// dst = order ? order[i] : i.  An entry packs the sub-state (low 32 bits)
// and 2 slot + (sign < 0) (high 32 bits).
template <typename R, int J>
__global__ void __launch_bounds__(256) k_psi(int P, int s0, int s1, const int* __restrict__ order,
                                             const int* __restrict__ eptr,
                                             const unsigned long long* __restrict__ ent,
                                             const R* __restrict__ tl, R tsign, R* __restrict__ psi) {
  int i = s0 + (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (i >= s1) return;
  int p = blockIdx.y * 32 * J + (threadIdx.x & 31);
  R acc[J];
#pragma unroll
  for (int j = 0; j < J; ++j) acc[j] = R(0);
  int e1 = eptr[i + 1];
  for (int e = eptr[i]; e < e1; ++e) {
    unsigned long long w = ent[e];
    unsigned sub = (unsigned)w, sl = (unsigned)(w >> 32);
    const R* a = tl + (size_t)(sl >> 1) * P + p;
    const R* b = psi + (size_t)sub * P + p;
    if (sl & 1) {
#pragma unroll
      for (int j = 0; j < J; ++j) acc[j] -= a[32 * j] * b[32 * j];
    } else {
#pragma unroll
      for (int j = 0; j < J; ++j) acc[j] += a[32 * j] * b[32 * j];
    }
  }
  R* d = psi + (size_t)(order ? order[i] : i) * P + p;
#pragma unroll
  for (int j = 0; j < J; ++j) d[32 * j] = tsign * acc[j];
}

// phi[o][p] = <out o| H |psi> - E_0 psi[o], E_0 = <ref|H|ref>: the rows off
// the diagonal in R, the diagonal and E_0 in FP64 from the same integrals (in
// FP32 their large common part then cancels exactly).  Off-diagonal entries
// are grouped by state s within a row and packed: s (bits 0-19), key slot
// (20-34), negative (35), coefficient 1/2 instead of 1 (36), first entry of
// a state (37); a run sums c v[key] and multiplies psi[s] once.
constexpr int kHsBits = 20, kHkBits = 15;
constexpr int kHNeg = kHsBits + kHkBits, kHHalf = kHNeg + 1, kHNew = kHNeg + 2;
template <typename R, int J>
__global__ void __launch_bounds__(256) k_phi(int P, int nout, const int* __restrict__ hptr,
                                             const unsigned long long* __restrict__ hent,
                                             const int* __restrict__ dptr, const int16_t* __restrict__ dkey,
                                             const double* __restrict__ dc, const double* __restrict__ e0,
                                             const R* __restrict__ vl, const R* __restrict__ psi,
                                             const int* __restrict__ out_state, R* __restrict__ phi) {
  int o = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (o >= nout) return;
  int p = blockIdx.y * 32 * J + (threadIdx.x & 31);
  double dg[J];
#pragma unroll
  for (int j = 0; j < J; ++j) dg[j] = -e0[p + 32 * j];
  int d1 = dptr[o + 1];
  for (int e = dptr[o]; e < d1; ++e) {
    const R* v = vl + (size_t)dkey[e] * P + p;
#pragma unroll
    for (int j = 0; j < J; ++j) dg[j] += dc[e] * double(v[32 * j]);
  }
  R acc[J], run[J];
#pragma unroll
  for (int j = 0; j < J; ++j) { acc[j] = R(0); run[j] = R(0); }
  const R* ps = psi + p;
  int e1 = hptr[o + 1];
  for (int e = hptr[o]; e < e1; ++e) {
    unsigned long long w = hent[e];
    if ((w >> kHNew) & 1) {
#pragma unroll
      for (int j = 0; j < J; ++j) { acc[j] += run[j] * ps[32 * j]; run[j] = R(0); }
      ps = psi + (size_t)(w & ((1u << kHsBits) - 1)) * P + p;
    }
    const R* v = vl + (size_t)((w >> kHsBits) & ((1u << kHkBits) - 1)) * P + p;
    R c = ((w >> kHHalf) & 1) ? R(0.5) : R(1);
    if ((w >> kHNeg) & 1) c = -c;
#pragma unroll
    for (int j = 0; j < J; ++j) run[j] += c * v[32 * j];
  }
  const R* pd = psi + (size_t)out_state[o] * P + p;
  R* out = phi + (size_t)o * P + p;
#pragma unroll
  for (int j = 0; j < J; ++j) out[32 * j] = acc[j] + run[j] * ps[32 * j] + R(dg[j] * double(pd[32 * j]));
}

// R_loc[subset][o] = sum sign psi_minus(w) phi(kappa); E_loc[subset] = phi(ref)
template <typename R, int J>
__global__ void __launch_bounds__(256) k_backsub(int P, int p0, int nsub, int nout, const int* __restrict__ bptr,
                                                 const int* __restrict__ bk, const int* __restrict__ bw,
                                                 const R* __restrict__ psim, const R* __restrict__ phi,
                                                 double* __restrict__ Rloc, double* __restrict__ Eloc) {
  int o = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  int p = blockIdx.y * 32 * J + (threadIdx.x & 31);
  if (o >= nout) return;
  if (o == 0) {
#pragma unroll
    for (int j = 0; j < J; ++j)
      if (p0 + p + 32 * j < nsub) Eloc[p0 + p + 32 * j] = double(phi[p + 32 * j]);
    return;
  }
  R acc[J];
#pragma unroll
  for (int j = 0; j < J; ++j) acc[j] = R(0);
  int e1 = bptr[o + 1];
  for (int e = bptr[o]; e < e1; ++e) {
    int w = bw[e];
    const R* a = psim + (size_t)(w >> 1) * P + p;
    const R* b = phi + (size_t)bk[e] * P + p;
    if (w & 1) {
#pragma unroll
      for (int j = 0; j < J; ++j) acc[j] -= a[32 * j] * b[32 * j];
    } else {
#pragma unroll
      for (int j = 0; j < J; ++j) acc[j] += a[32 * j] * b[32 * j];
    }
  }
#pragma unroll
  for (int j = 0; j < J; ++j)
    if (p0 + p + 32 * j < nsub) Rloc[(size_t)(p0 + p + 32 * j) * nout + o] = double(acc[j]);
}

// ------------------------------------------------------------ assembly
struct AsmArgs {
  const double* Rloc[kMaxSites + 1];  // [subset][output]
  int nsub[kMaxSites + 1];
  int nout[kMaxSites + 1];
  double c[kMaxSites + 1];
  int kmax;
};

// colex rank of a sorted label set
__device__ __forceinline__ int colex_d(const int* p, int m) {
  int r = 0;
  for (int i = 0; i < m; ++i) r += c_binom[p[i] * 8 + i + 1];
  return r;
}

// sum over the k-subsets L containing the sorted labels M (m <= 4 of them)
// of X[rank(L) * ld + base + colex(positions of M in L) * nper + j]; the
// subsets in a fixed order (the added labels in lexicographic order)
__device__ double superset_sum(int N, const int* M, int m, int k, const double* __restrict__ X, int ld, int base,
                               int nper, int j) {
  int nc = N - m, na = k - m;
  int e[kMaxSites];
  for (int x = 0; x < na; ++x) e[x] = x;
  double part = 0.0;
  for (;;) {
    // L = M + the e-th labels not in M (both sorted), merged
    int Ls[kMaxSites], pos[4], El[kMaxSites];
    for (int x = 0; x < na; ++x) {
      int lab = e[x];
      for (int y = 0; y < m; ++y)
        if (M[y] <= lab) ++lab;
      El[x] = lab;
    }
    int nl = 0, im = 0, ie = 0;
    while (nl < k) {
      if (im < m && (ie >= na || M[im] < El[ie])) { pos[im] = nl; Ls[nl++] = M[im++]; }
      else Ls[nl++] = El[ie++];
    }
    part += X[(size_t)colex_d(Ls, k) * ld + base + colex_d(pos, m) * nper + j];
    // next combination of na among nc (lexicographic)
    int x = na - 1;
    while (x >= 0 && e[x] == nc - na + x) --x;
    if (x < 0) break;
    ++e[x];
    for (int y = x + 1; y < na; ++y) e[y] = e[y - 1] + 1;
  }
  return part;
}

// r at the unique slots of m-label outputs: sum over subsets L containing the
// labels, |L| = k <= kmax, of c_k R_loc^(L); subsets in a fixed order
__global__ void k_assemble(int N, int m, int nch, const int8_t* __restrict__ subs_m, int nsets, AsmArgs A,
                           double* __restrict__ r) {
  size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (size_t)nsets * nch) return;
  int set = tid / nch, ch = tid % nch;
  int M[3];
  for (int x = 0; x < m; ++x) M[x] = subs_m[(size_t)set * m + x];
  double acc = 0.0;
  for (int k = m; k <= A.kmax; ++k) {
    if (A.c[k] == 0.0 || A.nsub[k] == 0) continue;
    int base = 1 + (m >= 2 ? 3 * k : 0) + (m >= 3 ? 29 * c_binom[k * 8 + 2] : 0);
    acc += A.c[k] * superset_sum(N, M, m, k, A.Rloc[k], A.nout[k], base, nch, ch);
  }
  size_t idx;
  if (m == 1) idx = 3 * (size_t)M[0] + ch;
  else if (m == 2) idx = 3 * (size_t)N + ((size_t)M[0] * N + M[1]) * 29 + ch;
  else idx = off3(N) + (((size_t)M[0] * N + M[1]) * N + M[2]) * kNA3 + ch;
  r[idx] = acc;
}

// E_c = sum_k c^E_k sum_subsets E_loc (one block, fixed order)
__global__ void k_energy(AsmArgs A, double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int k = 1; k <= A.kmax; ++k) {
    if (A.c[k] == 0.0) continue;
    double part = 0.0;
    for (int i = threadIdx.x; i < A.nsub[k]; i += blockDim.x) part += A.Rloc[k][i];
    s += A.c[k] * part;
  }
  s = ppq::block_sum(s, red);
  if (threadIdx.x == 0) *out = s;
}

// the other stored orders of every two- and three-pair entry from the sorted one
__global__ void k_fill_copies(size_t L, int N, int K, double* __restrict__ v) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L || i < (size_t)3 * N) return;
  if (i < off3(N)) {
    size_t j = i - 3 * N;
    int ch = j % 29; size_t q = j / 29;
    int P = q / N, Q = q % N;
    if (P < Q) return;
    if (P == Q) { v[i] = 0.0; return; }
    int k2 = ppq_a2_swap[ch];
    v[i] = ppq_a2_swsg[ch] * v[3 * (size_t)N + ((size_t)Q * N + P) * 29 + k2];
    return;
  }
  size_t j = i - off3(N);
  int ch = j % kNA3; size_t q = j / kNA3;
  int l[3] = {(int)(q / ((size_t)N * N)), (int)((q / N) % N), (int)(q % N)};
  if (l[0] < l[1] && l[1] < l[2]) return;
  if (l[0] == l[1] || l[1] == l[2] || l[0] == l[2]) { v[i] = 0.0; return; }
  int mo[3] = {c_A3[3 * ch], c_A3[3 * ch + 1], c_A3[3 * ch + 2]};
  int sg = 1;
  for (int a = 0; a < 3; ++a)
    for (int b = a + 1; b < 3; ++b)
      if (l[a] > l[b] && (ppq_par[mo[a]] & ppq_par[mo[b]])) sg = -sg;
  // sort labels carrying their monomials
  int sl[3] = {l[0], l[1], l[2]}, sm[3] = {mo[0], mo[1], mo[2]};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 2 - a; ++b)
      if (sl[b] > sl[b + 1]) {
        int tl = sl[b]; sl[b] = sl[b + 1]; sl[b + 1] = tl;
        int tm = sm[b]; sm[b] = sm[b + 1]; sm[b + 1] = tm;
      }
  int c2 = c_A3inv[(sm[0] << 8) | (sm[1] << 4) | sm[2]];
  v[i] = sg * v[off3(N) + (((size_t)sl[0] * N + sl[1]) * N + sl[2]) * kNA3 + c2];
}

// ------------------------------------------------------------ solver kernels
// rows: 0 -> sum over active unique slots of x0^2; j >= 1 -> <e_slot[order[j-1]], e_slot[inew]>
__global__ void k_udots(size_t L, int N, int mr, const double* __restrict__ x0, int m,
                        const double* __restrict__ slots, size_t ld, const int* __restrict__ order, int inew,
                        double* __restrict__ part) {
  __shared__ double red[32];
  int row = blockIdx.y;
  const double* a;
  const double* b;
  if (row == 0) { a = x0; b = x0; }
  else { a = slots + (size_t)order[row - 1] * ld; b = slots + (size_t)inew * ld; }
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += (size_t)gridDim.x * blockDim.x)
    if (is_active(i, N, mr)) s += a[i] * b[i];
  s = ppq::block_sum(s, red);
  if (threadIdx.x == 0) part[(size_t)row * gridDim.x + blockIdx.x] = s;
}

// out[r] = sum of part[r][*] in a fixed order; out[rows] = *e (energy copy)
__global__ void k_rows(int nb, int rows, const double* __restrict__ part, const double* __restrict__ e,
                       double* __restrict__ out) {
  __shared__ double red[32];
  for (int r = 0; r < rows; ++r) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[(size_t)r * nb + i];
    s = ppq::block_sum(s, red);
    if (threadIdx.x == 0) out[r] = s;
    __syncthreads();
  }
  if (threadIdx.x == 0 && e) out[rows] = *e;
}

// zero the unique slots the excitation-rank mask drops
__global__ void k_mask_rank(size_t L, int N, int mr, double* __restrict__ t) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < L && is_unique(i, N) && !is_active(i, N, mr)) t[i] = 0.0;
}

// Jacobi step on the active unique slots: tn = t + r / D, en = r / D; zero
// elsewhere (copies, and slots the excitation-rank mask drops)
__global__ void k_jacobi3(size_t L, int N, int mr, const double* __restrict__ t, const double* __restrict__ r,
                          const double* __restrict__ fo, const double* __restrict__ fv, double shift,
                          double* __restrict__ tn, double* __restrict__ en) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L) return;
  if (!is_active(i, N, mr)) { tn[i] = 0.0; en[i] = 0.0; return; }
  double d = denom3(i, N, fo, fv, shift);
  double e = d != 0.0 ? r[i] / d : 0.0;
  tn[i] = t[i] + e;
  en[i] = e;
}

}  // namespace ph

namespace ph {

// ------------------------------------------------------------ host side
struct DevTables {
  int nstate = 0, nslot = 0, nout = 0, nkey = 0, ne0 = 0;
  unsigned long long *ent = nullptr, *oent = nullptr, *hent = nullptr;  // packed entries
  std::vector<double> lvl_ent, olvl_ent;  // recursion entries per level (algorithmic work)
  double nh = 0, nruns = 0, nd = 0, nb = 0;
  std::vector<int> lvl_ptr, olvl_ptr;
  int *ent_ptr = nullptr, *slot_desc = nullptr, *out_state = nullptr;
  int *olvl_order = nullptr, *oent_ptr = nullptr, *key_desc = nullptr;
  int *h_ptr = nullptr, *b_ptr = nullptr, *b_k = nullptr, *b_w = nullptr, *d_ptr = nullptr;
  int16_t *e0_key = nullptr, *d_key = nullptr;
  double *e0_cd = nullptr, *d_c = nullptr;
};

struct Ctx {
  int dev = -1;
  bool consts = false;
  std::map<int, DevTables*> tabs;  // key k * 16 + K * 4 + KH
  // subsets of every size (colex order), for the current N
  int subs_N = 0;
  int8_t* subs[kMaxSites + 1] = {};
  int nsub[kMaxSites + 1] = {};
  // gathered integrals
  int gN = 0;
  double *G1 = nullptr, *G2 = nullptr, *G3 = nullptr, *G4 = nullptr;
  int g4N = 0;
  // local-problem buffers
  size_t cap_psi = 0, cap_out = 0, cap_phi = 0, cap_tl = 0, cap_vl = 0;
  void *psi = nullptr, *psim = nullptr, *phi = nullptr, *tl = nullptr, *vl = nullptr;
  double* e0loc = nullptr;  // E_0 of every subset of the chunk
  size_t cap_e0 = 0;
  double* Rloc[kMaxSites + 1] = {};
  double* Eloc[kMaxSites + 1] = {};
  size_t cap_R[kMaxSites + 1] = {}, cap_E[kMaxSites + 1] = {};
  // solver state
  size_t cap_L = 0;
  int cap_diis = 0;
  double *t = nullptr, *r = nullptr, *slot_t = nullptr, *slot_e = nullptr;
  double *tb = nullptr, *r64 = nullptr, *rb = nullptr, *del = nullptr, *rho = nullptr;  // defect correction
  unsigned long long* amax = nullptr;
  double *B = nullptr, *coef = nullptr, *part = nullptr, *rows = nullptr, *e = nullptr;
  int* order = nullptr;
  double* host = nullptr;  // pinned scalars / order staging
  int n_launches = 0;
};

std::map<int, Ctx*> g_ph;

constexpr size_t kPsiBudget = (size_t)4 << 30;  // bytes of psi per chunk

int ph_consts(Ctx* c) {
  if (c->consts) return 0;
  const Algebra& A = algebra();
  int8_t a3[303 * 3];
  int16_t inv[4096];
  for (int i = 0; i < 4096; ++i) inv[i] = -1;
  for (int ch = 0; ch < (int)A.A3.size(); ++ch) {
    for (int x = 0; x < 3; ++x) a3[3 * ch + x] = (int8_t)A.A3[ch][x];
    inv[(A.A3[ch][0] << 8) | (A.A3[ch][1] << 4) | A.A3[ch][2]] = (int16_t)ch;
  }
  int8_t keys[4][576 * 5];
  memset(keys, 0, sizeof keys);
  for (int m = 1; m <= 4; ++m)
    for (int j = 0; j < A.nkey(m); ++j)
      for (int x = 0; x < 5; ++x) keys[m - 1][5 * j + x] = (int8_t)A.key[m][j][x];
  CK(cudaMemcpyToSymbol(c_A3, a3, sizeof a3));
  CK(cudaMemcpyToSymbol(c_A3inv, inv, sizeof inv));
  CK(cudaMemcpyToSymbol(c_key, keys, sizeof keys));
  int bn[128 * 8];
  for (int n = 0; n < 128; ++n)
    for (int r = 0; r < 8; ++r) bn[n * 8 + r] = binom(n, r);
  CK(cudaMemcpyToSymbol(c_binom, bn, sizeof bn));
  c->consts = true;
  return 0;
}

template <typename V>
int upload(V** dst, const std::vector<V>& v) {
  CK(cudaMalloc((void**)dst, std::max<size_t>(v.size(), 1) * sizeof(V)));
  if (!v.empty()) CK(cudaMemcpy(*dst, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice));
  return 0;
}

int dev_tables(Ctx* c, int k, int K, int KH, DevTables** out) {
  int key = k * 16 + K * 4 + KH;
  auto it = c->tabs.find(key);
  if (it != c->tabs.end()) { *out = it->second; return 0; }
  int rc;
  const Tables* T = host_tables(k, K, KH, &rc);
  if (!T) return fail(-5, "ph: table generation failed for %d sites (%d)", k, rc);
  DevTables* d = new DevTables();
  d->nstate = T->nstate; d->nslot = T->nslot; d->nout = T->nout; d->nkey = T->nkey;
  d->ne0 = (int)T->e0_c.size();
  d->lvl_ptr = T->lvl_ptr; d->olvl_ptr = T->olvl_ptr;
  for (size_t lv = 0; lv + 1 < T->lvl_ptr.size(); ++lv)
    d->lvl_ent.push_back((double)T->ent_ptr[T->lvl_ptr[lv + 1]] - T->ent_ptr[T->lvl_ptr[lv]]);
  for (size_t lv = 0; lv + 1 < T->olvl_ptr.size(); ++lv)
    d->olvl_ent.push_back((double)T->oent_ptr[T->olvl_ptr[lv + 1]] - T->oent_ptr[T->olvl_ptr[lv]]);
  d->nh = (double)T->h_s.size(); d->nd = (double)T->d_key.size(); d->nb = (double)T->b_k.size();
  // packed entries: recursion (sub | (2 slot + sign) << 32); Hamiltonian rows
  // grouped by state, (s, key, sign, half, first-of-state) in one word
  std::vector<unsigned long long> ent(T->ent_sub.size()), oent(T->oent_sub.size()), hent(T->h_s.size());
  for (size_t e = 0; e < ent.size(); ++e)
    ent[e] = (unsigned long long)(unsigned)T->ent_sub[e] | ((unsigned long long)(uint16_t)T->ent_slot[e] << 32);
  for (size_t e = 0; e < oent.size(); ++e)
    oent[e] = (unsigned long long)(unsigned)T->oent_sub[e] | ((unsigned long long)(uint16_t)T->oent_slot[e] << 32);
  if (T->nstate >= (1 << kHsBits) || T->nkey >= (1 << kHkBits))
    return fail(-5, "ph: table fields overflow for %d sites", k);
  std::vector<int> hptr(T->h_ptr);
  for (int o = 0; o < T->nout; ++o) {
    std::vector<std::pair<long long, double>> row;
    for (int e = T->h_ptr[o]; e < T->h_ptr[o + 1]; ++e)
      row.push_back({(long long)T->h_s[e] * 65536 + T->h_key[e], T->h_c[e]});
    std::sort(row.begin(), row.end());
    int prev = -1;
    for (size_t q = 0; q < row.size(); ++q) {
      int st = (int)(row[q].first / 65536), ky = (int)(row[q].first % 65536);
      double cv = row[q].second;
      if (fabs(cv) != 1.0 && fabs(cv) != 0.5)
        return fail(-5, "ph: unexpected Hamiltonian coefficient %g for %d sites", cv, k);
      unsigned long long w = (unsigned long long)st | ((unsigned long long)ky << kHsBits) |
                             ((unsigned long long)(cv < 0) << kHNeg) |
                             ((unsigned long long)(fabs(cv) == 0.5) << kHHalf) |
                             ((unsigned long long)(st != prev) << kHNew);
      hent[T->h_ptr[o] + q] = w;
      if (st != prev) d->nruns += 1;
      prev = st;
    }
  }
  if ((rc = upload(&d->ent_ptr, T->ent_ptr)) || (rc = upload(&d->ent, ent)) ||
      (rc = upload(&d->slot_desc, T->slot_desc)) ||
      (rc = upload(&d->out_state, T->out_state)) || (rc = upload(&d->olvl_order, T->olvl_order)) ||
      (rc = upload(&d->oent_ptr, T->oent_ptr)) || (rc = upload(&d->oent, oent)) ||
      (rc = upload(&d->key_desc, T->key_desc)) ||
      (rc = upload(&d->h_ptr, T->h_ptr)) || (rc = upload(&d->hent, hent)) || (rc = upload(&d->e0_key, T->e0_key)) ||
      (rc = upload(&d->e0_cd, T->e0_c)) || (rc = upload(&d->d_ptr, T->d_ptr)) || (rc = upload(&d->d_key, T->d_key)) ||
      (rc = upload(&d->d_c, T->d_c)) || (rc = upload(&d->b_ptr, T->b_ptr)) ||
      (rc = upload(&d->b_k, T->b_k)) || (rc = upload(&d->b_w, T->b_w))) {
    delete d;
    return rc;
  }
  c->tabs[key] = d;
  *out = d;
  return 0;
}

double moebius(int N, int k, int kmax) {
  double s = 0.0;
  for (int j = 0; j <= kmax - k; ++j) s += ((j & 1) ? -1.0 : 1.0) * binom(N - k, j);
  return s;
}

// every k-subset of N labels in colex order (rank = sum_i C(L_i, i + 1))
int ph_subsets(Ctx* c, int N) {
  if (c->subs_N == N) return 0;
  for (int k = 1; k <= kMaxSites; ++k) {
    if (c->subs[k]) cudaFree(c->subs[k]);
    c->subs[k] = nullptr;
    c->nsub[k] = 0;
    if (k > N) continue;
    int cnt = binom(N, k);
    std::vector<int8_t> v((size_t)cnt * k);
    std::vector<int> p(k);
    for (int i = 0; i < k; ++i) p[i] = i;
    for (;;) {
      int rk = colex_rank(p.data(), k);
      for (int i = 0; i < k; ++i) v[(size_t)rk * k + i] = (int8_t)p[i];
      int x = k - 1;
      while (x >= 0 && p[x] == N - k + x) --x;
      if (x < 0) break;
      ++p[x];
      for (int y = x + 1; y < k; ++y) p[y] = p[y - 1] + 1;
    }
    int rc = upload(&c->subs[k], v);
    if (rc) return rc;
    c->nsub[k] = cnt;
  }
  c->subs_N = N;
  return 0;
}

int grow_buf(void** p, size_t* cap, size_t bytes) {
  if (bytes <= *cap) return 0;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  CK(cudaMalloc(p, bytes));
  *cap = bytes;
  return 0;
}

// subsets per chunk for k sites: a multiple of mult, psi within the budget
int chunk_size(int nsub, int nstate, size_t elem, int mult) {
  size_t cap = kPsiBudget / ((size_t)nstate * elem);
  cap = std::max<size_t>(mult, cap / mult * mult);
  size_t need = ((size_t)nsub + mult - 1) / mult * mult;
  return (int)std::min(cap, need);
}

Ctx* ctx() {
  int dev = 0;
  cudaGetDevice(&dev);
  Ctx*& c = g_ph[dev];
  if (!c) { c = new Ctx(); c->dev = dev; }
  return c;
}

// psi and psi_minus level by level, phi, back-substitution for one chunk of
// subsets (J subsets per lane)
template <typename R, int J>
int local_problem(Ctx* c, DevTables* T, int P, int p0, int nsub, int k, cudaStream_t s, bool backsub = true) {
  const double nv = std::min(P, nsub - p0), es = sizeof(R);
  R* psi = (R*)c->psi;
  R* psim = (R*)c->psim;
  R* phi = (R*)c->phi;
  const R* tl = (const R*)c->tl;
  const R* vl = (const R*)c->vl;
  unsigned gy = (unsigned)(P / (32 * J));
  for (size_t lv = 1; lv + 1 < T->lvl_ptr.size(); ++lv) {
    int s0 = T->lvl_ptr[lv], s1 = T->lvl_ptr[lv + 1];
    if (s1 <= s0) continue;
    k_psi<R, J><<<dim3((unsigned)((s1 - s0 + 7) / 8), gy), 256, 0, s>>>(P, s0, s1, nullptr, T->ent_ptr, T->ent,
                                                                         tl, R(1), psi);
    c->n_launches++;
    g_prof.done("ph::k_psi (exp(T)|ref> level)", s, T->lvl_ent[lv] * (8.0 + 2 * es * nv) + (s1 - s0) * es * nv,
                2.0 * T->lvl_ent[lv] * nv);
  }
  for (size_t lv = 1; lv + 1 < T->olvl_ptr.size(); ++lv) {
    int s0 = T->olvl_ptr[lv], s1 = T->olvl_ptr[lv + 1];
    if (s1 <= s0) continue;
    k_psi<R, J><<<dim3((unsigned)((s1 - s0 + 7) / 8), gy), 256, 0, s>>>(P, s0, s1, T->olvl_order, T->oent_ptr,
                                                                         T->oent, tl, R(-1), psim);
    c->n_launches++;
    g_prof.done("ph::k_psi (exp(-T)|ref> on outputs)", s,
                T->olvl_ent[lv] * (8.0 + 2 * es * nv) + (s1 - s0) * es * nv, 2.0 * T->olvl_ent[lv] * nv);
  }
  dim3 go((unsigned)((T->nout + 7) / 8), gy);
  k_phi<R, J><<<go, 256, 0, s>>>(P, T->nout, T->h_ptr, T->hent, T->d_ptr, T->d_key, T->d_c, c->e0loc, vl, psi,
                                 T->out_state, phi);
  g_prof.done("ph::k_phi (<kappa|H|psi>)", s,
              T->nh * 8.0 + (T->nh + T->nruns + T->nd) * es * nv + T->nout * 2 * es * nv,
              2.0 * (T->nh + T->nruns + T->nd) * nv);
  c->n_launches++;
  if (!backsub) {
    CK(cudaGetLastError());
    return 0;
  }
  k_backsub<R, J><<<go, 256, 0, s>>>(P, p0, nsub, T->nout, T->b_ptr, T->b_k, T->b_w, psim, phi, c->Rloc[k],
                                     c->Eloc[k]);
  c->n_launches++;
  g_prof.done("ph::k_backsub", s, T->nb * (8.0 + 2 * es * nv) + T->nout * 8.0 * nv, 2.0 * T->nb * nv);
  CK(cudaGetLastError());
  return 0;
}

// one residual evaluation: r (unique slots assembled, copies filled) and
// e_dev (device scalar E_c) at layout amplitudes t (device, copies consistent)
template <typename R>
int residual(Ctx* c, int N, int K, int KH, const double* t, double* r, double* e_dev, cudaStream_t s) {
  int rc;
  int kfull = K + KH, kmax = std::min(kfull, N);
  AsmArgs A{}, AE{};
  A.kmax = kmax;
  AE.kmax = std::min(KH, N);
  for (int k = 1; k <= kmax; ++k) {
    double ck = moebius(N, k, kfull), ce = k <= KH ? moebius(N, k, KH) : 0.0;
    if (ck == 0.0 && ce == 0.0) continue;
    DevTables* T;
    if ((rc = dev_tables(c, k, K, KH, &T))) return rc;
    int nsub = c->nsub[k];
    int J = nsub >= 384 ? 4 : nsub >= 96 ? 2 : 1;
    int P = chunk_size(nsub, T->nstate, sizeof(R), 32 * J);
    if ((rc = grow_buf(&c->psi, &c->cap_psi, (size_t)T->nstate * P * sizeof(R)))) return rc;
    if ((rc = grow_buf(&c->psim, &c->cap_out, (size_t)T->nout * P * sizeof(R)))) return rc;
    if ((rc = grow_buf(&c->phi, &c->cap_phi, (size_t)T->nout * P * sizeof(R)))) return rc;
    if ((rc = grow_buf(&c->tl, &c->cap_tl, (size_t)T->nslot * P * sizeof(R)))) return rc;
    if ((rc = grow_buf(&c->vl, &c->cap_vl, (size_t)T->nkey * P * sizeof(R)))) return rc;
    if ((rc = grow_buf((void**)&c->e0loc, &c->cap_e0, (size_t)P * sizeof(double)))) return rc;
    if ((rc = grow_buf((void**)&c->Rloc[k], &c->cap_R[k], (size_t)T->nout * nsub * sizeof(double)))) return rc;
    if ((rc = grow_buf((void**)&c->Eloc[k], &c->cap_E[k], (size_t)nsub * sizeof(double)))) return rc;
    R* psi = (R*)c->psi;
    R* psim = (R*)c->psim;
    R* tl = (R*)c->tl;
    R* vl = (R*)c->vl;
    for (int p0 = 0; p0 < nsub; p0 += P) {
      size_t nt = (size_t)T->nslot * P, nk = (size_t)T->nkey * P;
      k_gather_amp<R><<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(P, p0, nsub, k, T->nslot, T->slot_desc,
                                                                   c->subs[k], N, t, tl);
      k_gather_int<R><<<(unsigned)((nk + 255) / 256), 256, 0, s>>>(P, p0, nsub, k, T->nkey, T->key_desc,
                                                                   c->subs[k], N, c->G1, c->G2, c->G3, c->G4, vl);
      k_set_ref<R><<<(P + 127) / 128, 128, 0, s>>>(P, psi, psim, T->ne0, T->e0_key, T->e0_cd, vl, c->e0loc);
      c->n_launches += 3;
      g_prof.done("ph::gather (amplitudes, integrals)", s, (double)(T->nslot + T->nkey) * P * (sizeof(R) + 8.0));
      if (J == 4) rc = local_problem<R, 4>(c, T, P, p0, nsub, k, s);
      else if (J == 2) rc = local_problem<R, 2>(c, T, P, p0, nsub, k, s);
      else rc = local_problem<R, 1>(c, T, P, p0, nsub, k, s);
      if (rc) return rc;
    }
    A.nout[k] = T->nout;
    A.Rloc[k] = c->Rloc[k]; A.nsub[k] = nsub; A.c[k] = ck;
    AE.Rloc[k] = c->Eloc[k]; AE.nsub[k] = nsub; AE.c[k] = ce;
  }
  size_t L = layout_len(N, K);
  CK(cudaMemsetAsync(r, 0, sizeof(double) * L, s));
  const int nch[4] = {0, 3, 29, kNA3};
  for (int m = 1; m <= std::min(K, N); ++m) {
    size_t nt = (size_t)c->nsub[m] * nch[m];
    k_assemble<<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(N, m, nch[m], c->subs[m], c->nsub[m], A, r);
    c->n_launches++;
    double terms = 0.0;
    for (int k = m; k <= kmax; ++k)
      if (A.c[k] != 0.0) terms += binom(N - m, k - m);
    g_prof.done("ph::k_assemble", s, (double)nt * (terms + 1) * 8.0, 2.0 * nt * terms);
  }
  k_energy<<<1, 256, 0, s>>>(AE, e_dev);
  k_fill_copies<<<(unsigned)((L + 255) / 256), 256, 0, s>>>(L, N, K, r);
  c->n_launches += 2;
  g_prof.done("ph::k_energy, k_fill_copies", s, 16.0 * L);
  CK(cudaGetLastError());
  return 0;
}

// stage the PH integrals (Fock, bare one-body part, gathers) for (N, K_H)
int stage_ph(Ctx* c, Workspace* w, const Problem& P, int KH, cudaStream_t s) {
  int rc;
  int N = P.N, n = P.n;
  if ((rc = ph_consts(c))) return rc;
  if ((rc = ph_subsets(c, N))) return rc;
  if (c->gN < N) {
    if (c->G1) cudaFree(c->G1);
    if (c->G2) cudaFree(c->G2);
    if (c->G3) cudaFree(c->G3);
    CK(cudaMalloc((void**)&c->G1, sizeof(double) * N * 20));
    CK(cudaMalloc((void**)&c->G2, sizeof(double) * N * N * 232));
    CK(cudaMalloc((void**)&c->G3, sizeof(double) * N * N * N * kNK3));
    c->gN = N;
  }
  // K_H >= 3 keeps every (pq|ii), so the bare one-body part is h itself; for
  // K_H = 2 it is h' = f - sum_i [2 v'(pq|ii) - v'(pi|iq)] (staged by the PQ path)
  if (KH >= 4 && N >= 4 && c->g4N != N) {
    if (c->G4) cudaFree(c->G4);
    c->G4 = nullptr;
    CK(cudaMalloc((void**)&c->G4, sizeof(double) * c->nsub[4] * kNK4));
    c->g4N = N;
  }
  const double* hb = KH >= 3 ? P.h : w->hp;
  size_t nq = KH >= 4 && N >= 4 ? (size_t)c->nsub[4] : 0;
  size_t tot = (size_t)N * 20 + (size_t)N * N * 232 + (KH >= 3 ? (size_t)N * N * N * kNK3 : 0) + nq * kNK4;
  k_stage_g<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, N, KH, hb, P.src(), w->occ, w->vir, c->subs[4], (int)nq,
                                                          c->G1, c->G2, c->G3, c->G4);
  CK(cudaGetLastError());
  return 0;
}

int grow_solver(Ctx* c, size_t L, int diis) {
  if (L <= c->cap_L && diis <= c->cap_diis && c->host) return 0;
  size_t Lc = std::max(L, c->cap_L);
  int dc = std::max(diis, c->cap_diis);
  void* ps[] = {c->t, c->r, c->slot_t, c->slot_e, c->B, c->coef, c->part, c->rows, c->e, c->order,
                c->tb, c->r64, c->rb, c->del, c->rho, c->amax};
  for (void* p : ps)
    if (p) cudaFree(p);
  if (c->host) cudaFreeHost(c->host);
  CK(cudaMalloc((void**)&c->t, sizeof(double) * Lc));
  CK(cudaMalloc((void**)&c->r, sizeof(double) * Lc));
  for (double** b : {&c->tb, &c->r64, &c->rb, &c->del, &c->rho}) CK(cudaMalloc((void**)b, sizeof(double) * Lc));
  CK(cudaMalloc((void**)&c->amax, sizeof(unsigned long long)));
  CK(cudaMalloc((void**)&c->slot_t, sizeof(double) * Lc * std::max(dc, 1)));
  CK(cudaMalloc((void**)&c->slot_e, sizeof(double) * Lc * std::max(dc, 1)));
  CK(cudaMalloc((void**)&c->B, sizeof(double) * kDiisMax * kDiisMax));
  CK(cudaMalloc((void**)&c->coef, sizeof(double) * kDiisMax));
  CK(cudaMalloc((void**)&c->part, sizeof(double) * kRedBlocks * (kDiisMax + 2)));
  CK(cudaMalloc((void**)&c->rows, sizeof(double) * (kDiisMax + 4)));
  CK(cudaMalloc((void**)&c->e, sizeof(double) * 4));
  CK(cudaMalloc((void**)&c->order, sizeof(int) * kDiisMax));
  CK(cudaMallocHost((void**)&c->host, sizeof(double) * 64));
  c->cap_L = Lc;
  c->cap_diis = dc;
  return 0;
}

int residual_any(Ctx* c, int N, int K, int KH, int prec, const double* t, double* r, double* e, cudaStream_t s) {
  return prec ? residual<float>(c, N, K, KH, t, r, e, s) : residual<double>(c, N, K, KH, t, r, e, s);
}

}  // namespace ph

namespace ph {

// one residual evaluation through the C ABI: stage, copy t (sorted-label
// entries; copies filled), evaluate, copy r and E_c out
int residual_entry(int K, int KH, int n_pairs, const int* occ_of_pair, const int* vir_of_pair, const double* h,
                   const double* eri, const double* t, double* r, double* e_corr, int precision, cudaStream_t s) {
  if (precision != 0 && precision != 1) return fail(-4, "precision must be 0 or 1");
  if (!t || !r) return fail(-2, "t and r must be non-null");
  if (n_pairs > 127) return fail(-1, "n_pairs must be <= 127 for the label-subset residual");
  Workspace* w = nullptr;
  Problem P;
  int rc = prepare(n_pairs, occ_of_pair, vir_of_pair, h, eri, 1, s, &w, &P);
  if (rc) return rc;
  Ctx* c = ctx();
  if ((rc = stage_ph(c, w, P, KH, s))) return rc;
  int N = n_pairs;
  size_t L = layout_len(N, K);
  if ((rc = grow_solver(c, L, 1))) return rc;
  CK(cudaMemcpyAsync(c->t, t, sizeof(double) * L, cudaMemcpyDefault, s));
  k_fill_copies<<<(unsigned)((L + 255) / 256), 256, 0, s>>>(L, N, K, c->t);
  if ((rc = residual_any(c, N, K, KH, precision, c->t, c->r, c->e, s))) return rc;
  CK(cudaMemcpyAsync(r, c->r, sizeof(double) * L, cudaMemcpyDefault, s));
  CK(cudaMemcpyAsync(c->host, c->e, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (e_corr) *e_corr = c->host[0];
  return 0;
}

}  // namespace ph

extern "C" {

int ph_residual(int n_pairs, const int* occ_of_pair, const int* vir_of_pair, const double* h, const double* eri,
                const double* t, double* r, double* e_corr, int precision, int K_H, void* stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_err.clear();
  int KH = K_H == 0 ? 3 : K_H;
  if (KH != 2 && KH != 3) return fail(-4, "ph_residual: K_H must be 0, 2 or 3");
  return ph::residual_entry(3, KH, n_pairs, occ_of_pair, vir_of_pair, h, eri, t, r, e_corr, precision,
                            (cudaStream_t)stream);
}

}  // extern "C"

namespace ph {

// algorithmic work of one residual: 2 FLOPs per table entry and subset
// (recursions, Hamiltonian rows, back-substitution), over the subsets that
// enter with a nonzero coefficient
double residual_flops(int N, int K, int KH) {
  int kfull = K + KH;
  double f = 0.0;
  for (int k = 1; k <= std::min(kfull, N); ++k) {
    if (moebius(N, k, kfull) == 0.0 && (k > KH || moebius(N, k, KH) == 0.0)) continue;
    int rc;
    const Tables* T = host_tables(k, K, KH, &rc);
    if (!T) return 0.0;
    double per = 2.0 * ((double)T->ent_sub.size() + (double)T->oent_sub.size() + (double)T->h_s.size() +
                        (double)T->d_key.size() + (double)T->b_k.size());
    f += per * binom(N, k);
  }
  return f;
}

struct PhSolver {
  Ctx* c;
  int N, K, KH;
  size_t L;
  ppq_opts o;
  cudaStream_t s;
  Workspace* w;
  unsigned lb;
  int evals = 0, evals32 = 0;
  double t_res_ms = 0.0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<int> ring;  // slot ids, oldest first
  PhSolver(Ctx* c_, Workspace* w_, int N_, int K_, int KH_, const ppq_opts& o_, cudaStream_t s_)
      : c(c_), N(N_), K(K_), KH(KH_), L(layout_len(N_, K_)), o(o_), s(s_), w(w_), lb((unsigned)((L + 255) / 256)) {}
  ~PhSolver() {
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
  }
  int init() {
    CK(cudaEventCreate(&ev0));
    CK(cudaEventCreate(&ev1));
    return 0;
  }
  int eval(int prec, double* res, double* e) {
    CK(cudaEventRecord(ev0, s));
    int rc = residual_any(c, N, K, KH, prec, c->t, c->r, c->e, s);
    if (rc) return rc;
    CK(cudaEventRecord(ev1, s));
    k_udots<<<dim3(kRedBlocks, 1), 256, 0, s>>>(L, N, o.max_rank, c->r, 0, c->slot_e, L, c->order, 0, c->part);
    k_rows<<<1, 256, 0, s>>>(kRedBlocks, 1, c->part, c->e, c->rows);
    CK(cudaMemcpyAsync(c->host, c->rows, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
    g_prof.done("solver: norm, energy, device-to-host", s, 8.0 * L);
    CK(cudaStreamSynchronize(s));
    c->n_launches += 2;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    t_res_ms += ms;
    evals++;
    if (prec) evals32++;
    *res = sqrt(c->host[0]);
    *e = c->host[1];
    if (trace_on())
      fprintf(stderr, "ph eval %4d %s |R| %.3e E_c %.12f (%.2f ms)\n", evals, prec ? "fp32" : "fp64", *res, *e, ms);
    return 0;
  }
  // Jacobi step x + res/D on the unique slots, Pulay DIIS over `ring` (device)
  int step_on(double* x, const double* res, int it, std::vector<int>& rg) {
    int m_max = o.diis_dim > 0 ? o.diis_dim : 1;
    int slot = (int)rg.size() < m_max ? (int)rg.size() : rg.front();
    std::vector<int> act;
    for (int id : rg)
      if (id != slot) act.push_back(id);
    if ((int)act.size() >= m_max) act.erase(act.begin());
    act.push_back(slot);
    rg = act;
    int m = (int)act.size();
    double* st = c->slot_t + (size_t)slot * L;
    double* se = c->slot_e + (size_t)slot * L;
    k_jacobi3<<<lb, 256, 0, s>>>(L, N, o.max_rank, x, res, w->fo, w->fv, o.level_shift, st, se);
    int* ho = (int*)(c->host + 32);
    for (int i = 0; i < m; ++i) ho[i] = act[i];
    CK(cudaMemcpyAsync(c->order, ho, sizeof(int) * m, cudaMemcpyHostToDevice, s));
    k_udots<<<dim3(kRedBlocks, 1 + m), 256, 0, s>>>(L, N, o.max_rank, se, m, c->slot_e, L, c->order, slot,
                                                   c->part);
    k_rows<<<1, 256, 0, s>>>(kRedBlocks, 1 + m, c->part, nullptr, c->rows);
    int extrap = o.diis_dim > 0 && it >= o.diis_start && m > 1;
    k_diis_solve<<<1, 32, 0, s>>>(m, c->order, slot, c->rows, c->B, kDiisMax, extrap, c->coef);
    k_extrap<<<lb, 256, 0, s>>>(L, m, c->coef, c->slot_t, L, c->order, x);
    c->n_launches += 5;
    g_prof.done("solver: Jacobi, DIIS (device solve), extrapolation", s, 8.0 * L * (4 + 2 * m));
    CK(cudaGetLastError());
    return 0;
  }
  int step(int it) {
    int rc = step_on(c->t, c->r, it, ring);
    if (rc) return rc;
    k_fill_copies<<<lb, 256, 0, s>>>(L, N, K, c->t);
    c->n_launches++;
    return 0;
  }
  // weighted norm of x over the unique slots (host value)
  int norm(const double* x, double* out) {
    k_udots<<<dim3(kRedBlocks, 1), 256, 0, s>>>(L, N, o.max_rank, x, 0, c->slot_e, L, c->order, 0, c->part);
    k_rows<<<1, 256, 0, s>>>(kRedBlocks, 1, c->part, nullptr, c->rows);
    CK(cudaMemcpyAsync(c->host, c->rows, sizeof(double), cudaMemcpyDeviceToHost, s));
    g_prof.done("solver: norm, energy, device-to-host", s, 8.0 * L);
    CK(cudaStreamSynchronize(s));
    c->n_launches += 2;
    *out = sqrt(c->host[0]);
    return 0;
  }
  // FP64 defect correction (the polish of the mixed form): c->r holds R_64(t)
  // on entry.  Solves r + J d = 0 to a relative 1e-3 with DIIS-accelerated
  // Jacobi, Jacobian products by forward differences of FP32 residuals, then
  // t <- t + d.  The step is eta = 1e-2 in max norm: the FP32 residual of the
  // label-subset expansion carries a noise floor of ~1e-5 (inclusion-exclusion
  // coefficients of hundreds), which a smaller step would not rise above.
  int defect_correction(double r0, int* it_io) {
    const double eta = 1e-2, tol = 1e-3;
    int rc;
    CK(cudaMemcpyAsync(c->tb, c->t, sizeof(double) * L, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(c->r64, c->r, sizeof(double) * L, cudaMemcpyDeviceToDevice, s));
    double rn, ed;
    if ((rc = eval(1, &rn, &ed))) return rc;
    CK(cudaMemcpyAsync(c->rb, c->r, sizeof(double) * L, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(c->del, 0, sizeof(double) * L, s));
    CK(cudaMemcpyAsync(c->rho, c->r64, sizeof(double) * L, cudaMemcpyDeviceToDevice, s));
    std::vector<int> inner_ring;
    std::vector<double> hist;
    for (int inner = 0; inner < 30 && *it_io < o.max_iter; ++inner) {
      if ((rc = step_on(c->del, c->rho, inner + 1, inner_ring))) return rc;
      CK(cudaMemsetAsync(c->amax, 0, sizeof(unsigned long long), s));
      k_absmax<<<kRedBlocks, 256, 0, s>>>(L, c->del, c->amax);
      k_fd_point<<<lb, 256, 0, s>>>(L, c->tb, c->del, c->amax, eta, c->t);
      if ((rc = eval(1, &rn, &ed))) return rc;
      k_fd_rho<<<lb, 256, 0, s>>>(L, c->r64, c->r, c->rb, c->amax, eta, c->rho);
      c->n_launches += 3;
      g_prof.done("solver: defect-correction vectors", s, 8.0 * L * 6);
      (*it_io)++;
      double rr;
      if ((rc = norm(c->rho, &rr))) return rc;
      if (trace_on()) fprintf(stderr, "ph   inner %2d |r + J d| %.3e (target %.3e)\n", inner, rr, tol * r0);
      if (!isfinite(rr)) break;
      if (rr <= tol * r0) break;
      hist.push_back(rr);
      size_t k = hist.size();
      if (k >= 4 && hist[k - 1] > 0.9 * hist[k - 4]) break;
    }
    k_axpy_to<<<lb, 256, 0, s>>>(L, c->tb, c->del, c->t);
    k_fill_copies<<<lb, 256, 0, s>>>(L, N, K, c->t);
    c->n_launches += 2;
    CK(cudaGetLastError());
    return 0;
  }
};

}  // namespace ph

namespace {

// The K-pair model (K = 2 or 3) with integrals over at most KH labels (4 =
// untruncated) solved through the label-subset residual: Jacobi steps with
// orbital-energy denominators and device-side Pulay DIIS; the mixed form runs
// FP32 residuals until switch_tol (or FP32 stagnation), then FP64.
int subset_solve(int K, int KH, int n_pairs, const int* occ_of_pair, const int* vir_of_pair, const double* h,
                 const double* eri, const double* B, int naux, double e_const, const ppq_opts& o,
                 const double* t_in, double* t_out, double* e_corr, double* e_total, ppq_info* info,
                 cudaStream_t s, std::chrono::steady_clock::time_point wall0) {
  if (o.precision != 0 && o.precision != 1) return fail(-4, "precision must be 0 or 1");
  if (o.max_iter < 1 || o.diis_dim < 0 || o.diis_dim > kDiisMax)
    return fail(-4, "max_iter >= 1 and 0 <= diis_dim <= %d required", kDiisMax);
  if (o.guess == 1 && !t_in) return fail(-2, "guess = 1 needs t_in");
  if (o.max_rank < 0 || o.max_rank > 2 * K) return fail(-4, "max_rank must be 0 (every rank) or 1..%d", 2 * K);
  if (n_pairs > 127) return fail(-1, "n_pairs must be <= 127 for the label-subset solver");
  Workspace* w = nullptr;
  Problem P;
  int rc = B ? prepare_cd(n_pairs, occ_of_pair, vir_of_pair, h, B, naux, 1, s, &w, &P)
             : prepare(n_pairs, occ_of_pair, vir_of_pair, h, eri, 1, s, &w, &P);
  if (rc) {
    if (rc == 3 && info) { memset(info, 0, sizeof *info); info->status = 3; }
    return rc;
  }
  ph::Ctx* c = ph::ctx();
  c->n_launches = 0;
  g_prof.reset(o.profile != 0);
  struct ProfOff { ~ProfOff() { g_prof.on = false; } } prof_off;
  g_prof.start(s);
  if ((rc = ph::stage_ph(c, w, P, KH, s))) return rc;
  g_prof.done("staging (Fock, gathers)", s);
  int N = n_pairs, n = 2 * N;
  size_t L = ph::layout_len(N, K);
  int m_max = o.diis_dim > 0 ? o.diis_dim : 1;
  if ((rc = ph::grow_solver(c, L, m_max))) return rc;
  if (o.guess == 1) {
    CK(cudaMemcpyAsync(c->t, t_in, sizeof(double) * L, cudaMemcpyDefault, s));
    if (o.max_rank) ph::k_mask_rank<<<(unsigned)((L + 255) / 256), 256, 0, s>>>(L, N, o.max_rank, c->t);
    ph::k_fill_copies<<<(unsigned)((L + 255) / 256), 256, 0, s>>>(L, N, K, c->t);
  } else {
    CK(cudaMemsetAsync(c->t, 0, sizeof(double) * L, s));
  }
  k_eref<<<1, 1, 0, s>>>(N, n, P.h, w->f, w->occ, c->e + 1);
  CK(cudaMemcpyAsync(c->host + 40, c->e + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
  ph::PhSolver S(c, w, N, K, KH, o, s);
  if ((rc = S.init())) return rc;
  int prec = o.precision;
  int switched_at = prec ? -1 : 0;
  double e_old = 0.0, res = 0.0, e = 0.0;
  bool have_old = false;
  int status = 1, it;
  std::vector<double> hist;
  bool defect = false;  // FP64 defect-correction polish active
  double last_outer = 0.0;
  for (it = 1; it <= o.max_iter; ++it) {
    if (defect) {
      // one outer step: FP64 residual and test, then r + J d = 0 with FP32
      // finite-difference Jacobian products
      if ((rc = S.eval(0, &res, &e))) return rc;
      hist.push_back(res);
      if (!isfinite(res) || !isfinite(e) || res > 1e6) { status = 2; break; }
      if (have_old && res <= o.r_tol && fabs(e - e_old) <= o.e_tol) { status = 0; break; }
      bool stalled = last_outer > 0.0 && res > 0.1 * last_outer;
      e_old = e;
      have_old = true;
      if (stalled || res <= o.r_tol) {
        // the correction stopped paying, or only the energy test is left:
        // plain FP64 Jacobi/DIIS from here
        defect = false;
        S.ring.clear();
        if ((rc = S.step(it))) return rc;
        continue;
      }
      last_outer = res;
      if ((rc = S.defect_correction(res, &it))) return rc;
      continue;
    }
    if ((rc = S.eval(prec, &res, &e))) return rc;
    hist.push_back(res);
    if (!isfinite(res) || !isfinite(e) || res > 1e6) { status = 2; break; }
    if (prec == 0 && have_old && res <= o.r_tol && fabs(e - e_old) <= o.e_tol) { status = 0; break; }
    if (prec == 1) {
      // switch at switch_tol, or when FP32 stops gaining (< 10 % over three
      // steps below 1e-4: the FP32 noise floor)
      size_t k = hist.size();
      bool stagnant = k >= 4 && res < 1e-4 && hist[k - 1] > 0.9 * hist[k - 4];
      if (res <= (o.switch_tol > 0.0 ? o.switch_tol : 1e-5) || stagnant) {
        prec = 0;
        switched_at = it;
        have_old = false;
        S.ring.clear();
        if (o.polish == 1) defect = true;
        continue;  // re-evaluate at the same amplitudes in FP64
      }
    }
    e_old = e;
    have_old = true;
    if ((rc = S.step(it))) return rc;
  }
  if (it > o.max_iter) it = o.max_iter;
  if (t_out) CK(cudaMemcpyAsync(t_out, c->t, sizeof(double) * L, cudaMemcpyDefault, s));
  CK(cudaStreamSynchronize(s));
  double e_ref = c->host[40];
  if (e_corr) *e_corr = e;
  if (e_total) *e_total = e + e_ref + e_const;
  if (info) {
    memset(info, 0, sizeof *info);
    info->status = status;
    info->iters = S.evals;
    info->polish_iters = o.precision ? S.evals - S.evals32 : 0;
    info->switched_at = o.precision ? switched_at : -1;
    info->res_norm = res;
    info->e_corr = e;
    info->e_total = e + e_ref + e_const;
    info->t_residual_ms = S.t_res_ms;
    info->t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
    info->residual_flops = ph::residual_flops(N, K, KH);
    info->n_launches = c->n_launches + 10;
    info->evals_fp32 = S.evals32;
    info->evals_fp64 = S.evals - S.evals32;
  }
  return status;
}


}  // namespace

extern "C" {

int ph_solve(int n_pairs, const int* occ_of_pair, const int* vir_of_pair, const double* h,
             const double* eri, double e_const, const ppq_opts* opts, const double* t_in,
             double* t_out, double* e_corr, double* e_total, ppq_info* info, void* stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_err.clear();
  auto wall0 = std::chrono::steady_clock::now();
  ppq_opts o;
  if (opts) o = *opts; else ppq_default_opts(&o);
  int KH = o.K_H == 0 ? 3 : o.K_H;
  if (KH != 2 && KH != 3) return fail(-4, "ph_solve: K_H must be 0 (= 3), 2 or 3");
  return subset_solve(3, KH, n_pairs, occ_of_pair, vir_of_pair, h, eri, nullptr, 0, e_const, o, t_in, t_out, e_corr,
                      e_total, info, (cudaStream_t)stream, wall0);
}

int ph_solve_cd(int n_pairs, const int* occ_of_pair, const int* vir_of_pair, const double* h, const double* B,
                int naux, double e_const, const ppq_opts* opts, const double* t_in, double* t_out, double* e_corr,
                double* e_total, ppq_info* info, void* stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_err.clear();
  auto wall0 = std::chrono::steady_clock::now();
  ppq_opts o;
  if (opts) o = *opts; else ppq_default_opts(&o);
  int KH = o.K_H == 0 ? 3 : o.K_H;
  if (KH != 2 && KH != 3) return fail(-4, "ph_solve_cd: K_H must be 0 (= 3), 2 or 3");
  if (!B) return fail(-2, "B must be non-null");
  return subset_solve(3, KH, n_pairs, occ_of_pair, vir_of_pair, h, nullptr, B, naux, e_const, o, t_in, t_out,
                      e_corr, e_total, info, (cudaStream_t)stream, wall0);
}

int ppq_subset_residual(int K, int K_H, int n_pairs, const int* occ_of_pair, const int* vir_of_pair,
                        const double* h, const double* eri, const double* t, double* r, double* e_corr,
                        int precision, void* stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_err.clear();
  int KH = K_H == 0 ? K : (K_H < 0 ? 4 : K_H);
  if (K != 2 && K != 3) return fail(-4, "ppq_subset_residual: K must be 2 or 3");
  if (KH < 2 || KH > 4 || K + KH > ph::kMaxSites)
    return fail(-4, "ppq_subset_residual: K_H must be 0, 2, 3 or -1 (untruncated, K = 2 only)");
  return ph::residual_entry(K, KH, n_pairs, occ_of_pair, vir_of_pair, h, eri, t, r, e_corr, precision,
                            (cudaStream_t)stream);
}

}  // extern "C"
