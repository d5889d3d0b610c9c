// ph_adjoint.cuh -- the reverse pass of the label-subset residual: the PH
// Lagrangian gradient, the Lambda equations and the energy gradients with
// respect to the integrals and to orbital rotations; included after
// ph_engine.cuh.
//
// The Lagrangian of the projected equations (Theory section: lambda lives on
// the same truncated manifold as t),
//     L(t, lambda) = E_c(t) + sum over unique mu of lambda_mu R_mu(t),
// is by the label-subset expansion a weighted sum of local quantities,
//     L = sum_L [ c^E_|L| phi'_L(ref) + c_|L| sum_{o != ref} lambda_{mu(o)} R^(L)_o ],
// so its gradient is a sum over subsets of the reverse pass of each local
// problem, weights w_ref = c^E_k and w_o = c_k lambda_{mu(o)}:
//     phibar(kappa) = sum_o w_o sign psi_minus(u)         (back-substitution)
//     pmbar(u)      = sum_o w_o sign phi(kappa)  + reverse exp(-T) recursion
//     psibar(s)     = sum_kappa c v phibar(kappa) + (D - E_0) phibar   + reverse exp(T) recursion
//     tbar(slot)    = - sum sign psi_minus(sub) pmbar(u) + sum sign psi(sub) psibar(s)
//     vbar(key)     = sum c psi(s) phibar(kappa) + sum d psi(o) phibar(o) - dE_0/dv S,
//                     S = sum_o psi(o) phibar(o)
// from tables holding the forward entries grouped by their inputs
// (ph_tables.cuh, AdjTables).  Every adjoint is summed over the subsets that
// contain its labels (the transpose of the gathers) in a fixed order, so the
// gradient is reproducible; the integral adjoints then go through the
// transposed staging to dense dE/dh and dE/d(pq|rs).
#pragma once

namespace ph {

// ------------------------------------------------------------ kernels
// Entry lists longer than kSegLen are cut into segments: a warp sums one
// segment into part[segment][lane], a second kernel adds a row's segments in
// a fixed order.  The lists of the reverse pass are very uneven (a
// single-site amplitude occurs in up to 2.3e5 entries of a six-site sector,
// the reference state and output in 6.5e3), and a warp per whole row would
// wait on its longest row.
constexpr int kSegLen = 1024;

__device__ __forceinline__ size_t slot_index(int d, const int8_t* L, int N) {
  int m = d & 15, ch = d >> kDescIdx;
  size_t a = L[(d >> 4) & 15];
  if (m == 1) return 3 * a + ch;
  size_t b = L[(d >> 8) & 15];
  if (m == 2) return 3 * (size_t)N + (a * N + b) * 29 + ch;
  return off3(N) + ((a * N + b) * N + (size_t)L[(d >> 12) & 15]) * kNA3 + ch;
}

// weights of the local Lagrangian: wl[0][p] = c^E_k, wl[1 + slot][p] = c_k
// lambda at the slot's amplitude (the outputs after the reference are the
// slots, in the same order)
__global__ void k_gather_w(int P, int p0, int nsub, int k, int nslot, const int* __restrict__ slot_desc,
                           const int8_t* __restrict__ subs, int N, const double* __restrict__ lam, double ck,
                           double ce, double* __restrict__ wl) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)(nslot + 1) * P) return;
  int row = i / P, p = i % P;
  double v = 0.0;
  if (p0 + p < nsub) v = row == 0 ? ce : ck * lam[slot_index(slot_desc[row - 1], subs + (size_t)(p0 + p) * k, N)];
  wl[i] = v;
}

// one level of a reverse recursion (the rows of a level read only rows of
// higher levels, final before these launches), in segments: part[sg - sg0][p]
// = sum sign t[slot] x[s] over segment sg's entries (s | (2 slot + sign) << 32),
// the segments of the level's rows being [sg0, sg1)
template <int J>
__global__ void __launch_bounds__(256) k_rev_part(int P, int sg0, int sg1, const int* __restrict__ rng,
                                                  const unsigned long long* __restrict__ ent,
                                                  const double* __restrict__ tl, const double* __restrict__ x,
                                                  double* __restrict__ part) {
  int sg = sg0 + (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (sg >= sg1) return;
  int p = blockIdx.y * 32 * J + (threadIdx.x & 31);
  double acc[J];
#pragma unroll
  for (int j = 0; j < J; ++j) acc[j] = 0.0;
  for (int e = rng[2 * sg]; e < rng[2 * sg + 1]; ++e) {
    unsigned long long w = ent[e];
    unsigned sl = (unsigned)(w >> 32);
    const double* a = tl + (size_t)(sl >> 1) * P + p;
    const double* b = x + (size_t)(unsigned)w * P + p;
    double sgn = (sl & 1) ? -1.0 : 1.0;
#pragma unroll
    for (int j = 0; j < J; ++j) acc[j] += sgn * a[32 * j] * b[32 * j];
  }
#pragma unroll
  for (int j = 0; j < J; ++j) part[(size_t)(sg - sg0) * P + p + 32 * j] = acc[j];
}

// x[dst(i)] += tsign * (row i's segment sums, in order) for the rows [r0, r1)
__global__ void k_rev_sum(int P, int r0, int r1, const int* __restrict__ order, const int* __restrict__ segptr,
                          int sg0, const double* __restrict__ part, double tsign, double* __restrict__ x) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)(r1 - r0) * P) return;
  int i = r0 + (int)(t / P), p = t % P;
  int g0 = segptr[i], g1 = segptr[i + 1];
  if (g0 == g1) return;
  double acc = 0.0;
  for (int sg = g0; sg < g1; ++sg) acc += part[(size_t)(sg - sg0) * P + p];
  x[(size_t)(order ? order[i] : i) * P + p] += tsign * acc;
}

// the back-substitution in reverse, in segments: kind 0 (bit 31 clear) sums
// sign w[o] psi_minus(x) over entries of bk (-> phibar), kind 1 sums
// sign w[o] phi(x) over entries of bw (-> pmbar); entries o | x << 13 | sign << 26
template <int J>
__global__ void __launch_bounds__(256) k_adj_bsub_part(int P, int nseg, const int* __restrict__ seg_kind,
                                                       const int* __restrict__ rng, const unsigned* __restrict__ bk_ent,
                                                       const unsigned* __restrict__ bw_ent,
                                                       const double* __restrict__ wl, const double* __restrict__ pm,
                                                       const double* __restrict__ phi, double* __restrict__ part) {
  int sg = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (sg >= nseg) return;
  int p = blockIdx.y * 32 * J + (threadIdx.x & 31);
  const bool kw = seg_kind[sg] < 0;
  const unsigned* ent = kw ? bw_ent : bk_ent;
  const double* X = kw ? phi : pm;
  double acc[J];
#pragma unroll
  for (int j = 0; j < J; ++j) acc[j] = 0.0;
  for (int e = rng[2 * sg]; e < rng[2 * sg + 1]; ++e) {
    unsigned x = ent[e];
    const double* W = wl + (size_t)(x & 8191u) * P + p;
    const double* M = X + (size_t)((x >> 13) & 8191u) * P + p;
    double sgn = (x >> 26) & 1u ? -1.0 : 1.0;
#pragma unroll
    for (int j = 0; j < J; ++j) acc[j] += sgn * W[32 * j] * M[32 * j];
  }
#pragma unroll
  for (int j = 0; j < J; ++j) part[(size_t)sg * P + p + 32 * j] = acc[j];
}

// phibar[o] and pmbar[o] from their segment sums in order; the reference row
// of phibar adds w_ref (E_c takes phi'(ref) itself)
__global__ void k_adj_bsub_sum(int P, int nout, const int* __restrict__ kptr, const int* __restrict__ wptr,
                               const double* __restrict__ part, const double* __restrict__ wl,
                               double* __restrict__ phib, double* __restrict__ pmb) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)nout * P) return;
  int o = t / P, p = t % P;
  double a = o == 0 ? wl[p] : 0.0, b = 0.0;
  for (int sg = kptr[o]; sg < kptr[o + 1]; ++sg) a += part[(size_t)sg * P + p];
  for (int sg = wptr[o]; sg < wptr[o + 1]; ++sg) b += part[(size_t)sg * P + p];
  phib[(size_t)o * P + p] = a;
  pmb[(size_t)o * P + p] = b;
}

// psibar[s] before the reverse recursion, warp per sector state: the
// Hamiltonian rows read by state (kappa | key << 13 | neg << 28 | half << 29)
// and, for a state that is an output o, (D_o - E_0) phibar[o]
template <int J>
__global__ void __launch_bounds__(256) k_adj_rows(int P, int nstate, const int* __restrict__ hs_ptr,
                                                  const unsigned* __restrict__ hs_ent,
                                                  const int* __restrict__ out_of_state, const int* __restrict__ dptr,
                                                  const int16_t* __restrict__ dkey, const double* __restrict__ dc,
                                                  const double* __restrict__ e0, const double* __restrict__ vl,
                                                  const double* __restrict__ phib, double* __restrict__ psib) {
  int st = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (st >= nstate) return;
  int p = blockIdx.y * 32 * J + (threadIdx.x & 31);
  double acc[J];
#pragma unroll
  for (int j = 0; j < J; ++j) acc[j] = 0.0;
  for (int e = hs_ptr[st]; e < hs_ptr[st + 1]; ++e) {
    unsigned x = hs_ent[e];
    const double* v = vl + (size_t)((x >> 13) & 0x7FFFu) * P + p;
    const double* f = phib + (size_t)(x & 8191u) * P + p;
    double c = ((x >> 29) & 1u) ? 0.5 : 1.0;
    if ((x >> 28) & 1u) c = -c;
#pragma unroll
    for (int j = 0; j < J; ++j) acc[j] += c * v[32 * j] * f[32 * j];
  }
  int o = out_of_state[st];
  if (o >= 0) {
    double dg[J];
#pragma unroll
    for (int j = 0; j < J; ++j) dg[j] = -e0[p + 32 * j];
    for (int e = dptr[o]; e < dptr[o + 1]; ++e) {
      const double* v = vl + (size_t)dkey[e] * P + p;
#pragma unroll
      for (int j = 0; j < J; ++j) dg[j] += dc[e] * v[32 * j];
    }
    const double* f = phib + (size_t)o * P + p;
#pragma unroll
    for (int j = 0; j < J; ++j) acc[j] += dg[j] * f[32 * j];
  }
#pragma unroll
  for (int j = 0; j < J; ++j) psib[(size_t)st * P + p + 32 * j] = acc[j];
}

// tbar[slot] from the entries that read the slot's amplitude: the exp(-T)
// entries (s | sub << 20 | sign << 40, psi_minus = exp(-T)) and the exp(T)
// entries.  A slot's entry list is cut into segments of at most kSegLen
// entries (single-site amplitudes occur in up to 2.3e5 entries of a six-site
// sector, the mean is 7e3); warp per segment, the segment's partial sum to
// part[seg][p].  seg_slot packs the slot and (bit 31) exp(T) entries;
// seg_rng[2 seg], seg_rng[2 seg + 1] are the segment's first and end entry.
template <int J>
__global__ void __launch_bounds__(256) k_adj_tbar_part(int P, int nseg, const int* __restrict__ seg_slot,
                                                       const int* __restrict__ seg_rng,
                                                       const unsigned long long* __restrict__ obl_ent,
                                                       const unsigned long long* __restrict__ bl_ent,
                                                       const double* __restrict__ pm, const double* __restrict__ pmb,
                                                       const double* __restrict__ psi,
                                                       const double* __restrict__ psib, double* __restrict__ part) {
  int sg = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (sg >= nseg) return;
  int p = blockIdx.y * 32 * J + (threadIdx.x & 31);
  const bool fwd = seg_slot[sg] < 0;   // bit 31: exp(T) entries
  const int e0 = seg_rng[2 * sg], e1 = seg_rng[2 * sg + 1];
  const unsigned long long* ent = fwd ? bl_ent : obl_ent;
  const double* X = fwd ? psi : pm;
  const double* Xb = fwd ? psib : pmb;
  const double pos = fwd ? 1.0 : -1.0;   // psi_minus carries -T
  double acc[J];
#pragma unroll
  for (int j = 0; j < J; ++j) acc[j] = 0.0;
  for (int e = e0; e < e1; ++e) {
    unsigned long long w = ent[e];
    const double* a = X + (size_t)((w >> 20) & 0xFFFFFu) * P + p;
    const double* b = Xb + (size_t)(w & 0xFFFFFu) * P + p;
    double sgn = ((w >> 40) & 1u) ? -pos : pos;
#pragma unroll
    for (int j = 0; j < J; ++j) acc[j] += sgn * a[32 * j] * b[32 * j];
  }
#pragma unroll
  for (int j = 0; j < J; ++j) part[(size_t)sg * P + p + 32 * j] = acc[j];
}

// Tloc[subset][1 + slot] = the slot's segment sums in a fixed order
__global__ void k_adj_tbar_sum(int P, int p0, int nsub, int nslot, const int* __restrict__ seg_ptr,
                               const double* __restrict__ part, double* __restrict__ Tloc) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)nslot * P) return;
  int sl = i / P, p = i % P;
  if (p0 + p >= nsub) return;
  double acc = 0.0;
  for (int sg = seg_ptr[sl]; sg < seg_ptr[sl + 1]; ++sg) acc += part[(size_t)sg * P + p];
  Tloc[(size_t)(p0 + p) * (nslot + 1) + 1 + sl] = acc;
}

// S[p] = sum_o psi(state(o)) phibar(o): block per 32 subsets, 8 warps over
// the outputs, fixed-order reduction
__global__ void __launch_bounds__(256) k_adj_S(int P, int nout, const int* __restrict__ out_state,
                                               const double* __restrict__ psi, const double* __restrict__ phib,
                                               double* __restrict__ S) {
  __shared__ double red[8][32];
  int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  int p = blockIdx.x * 32 + lane;
  double s = 0.0;
  for (int o = wp; o < nout; o += 8) s += psi[(size_t)out_state[o] * P + p] * phib[(size_t)o * P + p];
  red[wp][lane] = s;
  __syncthreads();
  if (wp == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += red[q][lane];
    S[p] = t;
  }
}

// vbar[key] of every subset of the chunk, warp per key, stored as
// Vloc[subset][key]: off-diagonal rows by key (kappa | s << 13 | neg << 33 |
// half << 34), the diagonal by key, and E_0 through S
template <int J>
__global__ void __launch_bounds__(256) k_adj_vbar(int P, int p0, int nsub, int nkey, const int* __restrict__ hk_ptr,
                                                  const unsigned long long* __restrict__ hk_ent,
                                                  const int* __restrict__ dk_ptr, const int* __restrict__ dk_out,
                                                  const double* __restrict__ dk_c,
                                                  const double* __restrict__ e0_by_key,
                                                  const int* __restrict__ out_state, const double* __restrict__ psi,
                                                  const double* __restrict__ phib, const double* __restrict__ S,
                                                  double* __restrict__ Vloc) {
  int key = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (key >= nkey) return;
  int p = blockIdx.y * 32 * J + (threadIdx.x & 31);
  double acc[J];
  double ek = e0_by_key[key];
#pragma unroll
  for (int j = 0; j < J; ++j) acc[j] = -ek * S[p + 32 * j];
  for (int e = hk_ptr[key]; e < hk_ptr[key + 1]; ++e) {
    unsigned long long w = hk_ent[e];
    const double* a = psi + (size_t)((w >> 13) & 0xFFFFFu) * P + p;
    const double* b = phib + (size_t)(w & 8191u) * P + p;
    double c = ((w >> 34) & 1u) ? 0.5 : 1.0;
    if ((w >> 33) & 1u) c = -c;
#pragma unroll
    for (int j = 0; j < J; ++j) acc[j] += c * a[32 * j] * b[32 * j];
  }
  for (int e = dk_ptr[key]; e < dk_ptr[key + 1]; ++e) {
    int o = dk_out[e];
    const double* a = psi + (size_t)out_state[o] * P + p;
    const double* b = phib + (size_t)o * P + p;
    double c = dk_c[e];
#pragma unroll
    for (int j = 0; j < J; ++j) acc[j] += c * a[32 * j] * b[32 * j];
  }
#pragma unroll
  for (int j = 0; j < J; ++j)
    if (p0 + p + 32 * j < nsub) Vloc[(size_t)(p0 + p + 32 * j) * nkey + key] = acc[j];
}

// integral keys per label set: 20, 232, 576, 384 for 1..4 labels
__constant__ int c_nkey_m[5] = {0, 20, 232, 576, 384};

struct KeyAsm {
  const double* V[kMaxSites + 1];  // [subset][key]
  int nsub[kMaxSites + 1];
  int nkey[kMaxSites + 1];
  int kmax;
};

// dL/d(integral key j of the sorted label set M): the sum over subsets L
// containing M of vbar at the key's local index (keys of a k-site problem:
// by label count, then colex rank of the positions, then key index)
__global__ void k_assemble_keys(int N, int m, const int8_t* __restrict__ subs_m, int nsets, KeyAsm A,
                                double* __restrict__ out) {
  int nper = c_nkey_m[m];
  size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (size_t)nsets * nper) return;
  int set = tid / nper, j = tid % nper;
  int M[4];
  for (int x = 0; x < m; ++x) M[x] = subs_m[(size_t)set * m + x];
  double acc = 0.0;
  for (int k = m; k <= A.kmax; ++k) {
    if (A.nsub[k] == 0) continue;
    int base = 0;
    for (int q = 1; q < m; ++q) base += c_binom[k * 8 + q] * c_nkey_m[q];
    acc += superset_sum(N, M, m, k, A.V[k], A.nkey[k], base, nper, j);
  }
  out[tid] = acc;
}

// dL/dh' and dL/dv (dense, before the chain rule) from the key adjoints: the
// transpose of k_stage_g (orbitals occ[L_x], vir[L_x] of the sorted labels)
__global__ void k_scatter_keys(int n, int m, const int8_t* __restrict__ subs_m, int nsets,
                               const double* __restrict__ gb, const int* __restrict__ occ,
                               const int* __restrict__ vir, double* __restrict__ dh, double* __restrict__ dv) {
  int nper = c_nkey_m[m];
  size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (size_t)nsets * nper) return;
  double v = gb[tid];
  if (v == 0.0) return;
  int set = tid / nper, j = tid % nper;
  int o[8];
  for (int x = 0; x < m; ++x) {
    int L = subs_m[(size_t)set * m + x];
    o[2 * x] = occ[L];
    o[2 * x + 1] = vir[L];
  }
  const int8_t* k = c_key[m - 1] + 5 * j;
  size_t n1 = n, n2 = n1 * n, n3 = n2 * n;
  if (k[0] == 0) atomicAdd(&dh[o[k[1]] * n1 + o[k[2]]], v);
  else atomicAdd(&dv[o[k[1]] * n3 + o[k[2]] * n2 + o[k[3]] * n1 + o[k[4]]], v);
}

// ------------------------------------------------------------ host side
struct DevAdj {
  int *bs_ptr = nullptr, *bl_ptr = nullptr, *obs_ptr = nullptr, *obl_ptr = nullptr, *hs_ptr = nullptr;
  int *hk_ptr = nullptr, *dk_ptr = nullptr, *dk_out = nullptr, *bk_ptr = nullptr, *bw_ptr = nullptr;
  int* out_of_state = nullptr;
  unsigned long long *bs_ent = nullptr, *bl_ent = nullptr, *obs_ent = nullptr, *obl_ent = nullptr, *hk_ent = nullptr;
  unsigned *hs_ent = nullptr, *bk_ent = nullptr, *bw_ent = nullptr;
  double *dk_c = nullptr, *e0_by_key = nullptr;
  double nent = 0.0;                 // all entries (algorithmic work per subset)
  // segments of the by-slot entry lists (k_adj_tbar_part): slot (bit 31: exp(T)
  // entries), [first, end) entry, and the segments of each slot (CSR)
  int nseg = 0;
  int *seg_slot = nullptr, *seg_rng = nullptr, *seg_ptr = nullptr;
  // segments of the reverse recursions (rows in level order) and of the
  // back-substitution lists; the level ranges on the host
  int *rs_rng = nullptr, *rs_ptr = nullptr, *ro_rng = nullptr, *ro_ptr = nullptr;
  std::vector<int> rs_lvl, ro_lvl;
  int nbseg = 0;
  int *bseg_kind = nullptr, *bseg_rng = nullptr, *bk_segptr = nullptr, *bw_segptr = nullptr;
  size_t part_rows = 0;  // segments one launch writes at most (size of the partial buffer / P)
};

// segments of at most kSegLen entries of the rows [0, nrows) of a CSR list:
// entry ranges (rng, two ints each) and the rows' segments (ptr)
inline void segment_rows(const std::vector<int>& eptr, std::vector<int>& rng, std::vector<int>& ptr) {
  ptr.assign(1, 0);
  for (size_t i = 0; i + 1 < eptr.size(); ++i) {
    for (int e = eptr[i]; e < eptr[i + 1]; e += kSegLen) {
      rng.push_back(e);
      rng.push_back(std::min(e + kSegLen, eptr[i + 1]));
    }
    ptr.push_back((int)(rng.size() / 2));
  }
}

struct AdjCtx {
  std::map<int, DevAdj*> tabs;
  size_t cap_w = 0, cap_phib = 0, cap_pmb = 0, cap_psib = 0, cap_S = 0;
  double *wl = nullptr, *phib = nullptr, *pmb = nullptr, *psib = nullptr, *S = nullptr;
  double* part = nullptr;  // segment partial sums of tbar
  size_t cap_part = 0;
  double* Tloc[kMaxSites + 1] = {};
  double* Vloc[kMaxSites + 1] = {};
  size_t cap_T[kMaxSites + 1] = {}, cap_V[kMaxSites + 1] = {};
  double* Gb[5] = {};
  size_t cap_G[5] = {};
  size_t cap_L = 0;
  double *lam = nullptr, *grad = nullptr;
  size_t cap_n = 0;
  double *dhp = nullptr, *gh_raw = nullptr, *gh = nullptr, *gv_raw = nullptr, *gv = nullptr, *dk = nullptr,
         *ab = nullptr;
  // forward quantities of every chunk (psi, psi_minus, phi, t, v, E_0 per
  // subset) kept in HBM while t is fixed (the Lambda iterations, then the
  // integral gradients): a reverse pass then runs only the reverse kernels
  bool fwd_valid = false;
  int fwd_key = -1;
  void* fwd[kMaxSites + 1] = {};
  size_t fwd_cap[kMaxSites + 1] = {};
};

// bytes of the cached forward quantities of one chunk of P subsets of k sites
inline size_t fwd_chunk_bytes(const DevTables* T, int P) {
  return (size_t)(T->nstate + 2 * (size_t)T->nout + T->nslot + T->nkey + 1) * P * sizeof(double);
}

std::map<int, AdjCtx*> g_ph_adj;

AdjCtx* adj_ctx() {
  int dev = 0;
  cudaGetDevice(&dev);
  AdjCtx*& a = g_ph_adj[dev];
  if (!a) a = new AdjCtx();
  return a;
}

int dev_adjoint(AdjCtx* a, int k, int K, int KH, DevAdj** out) {
  int key = k * 16 + K * 4 + KH;
  auto it = a->tabs.find(key);
  if (it != a->tabs.end()) { *out = it->second; return 0; }
  int rc;
  const Tables* T = host_tables(k, K, KH, &rc);
  const AdjTables* A = T ? host_adjoint(k, K, KH, &rc) : nullptr;
  if (!A) return fail(-5, "ph: adjoint table generation failed for %d sites (%d)", k, rc);
  DevAdj* d = new DevAdj();
  d->nent = (double)A->bs_ent.size() + A->bl_ent.size() + A->obs_ent.size() + A->obl_ent.size() +
            A->hs_ent.size() + A->bk_ent.size() + A->bw_ent.size();
  {
    // per slot: segments of the exp(-T) entries, then of the exp(T) entries
    std::vector<int> ss, rng, sp(1, 0);
    for (int sl = 0; sl < T->nslot; ++sl) {
      for (int kind = 0; kind < 2; ++kind) {
        const std::vector<int>& ptr = kind ? A->bl_ptr : A->obl_ptr;
        for (int e = ptr[sl]; e < ptr[sl + 1]; e += kSegLen) {
          ss.push_back(kind ? (int)(sl | 0x80000000u) : sl);
          rng.push_back(e);
          rng.push_back(std::min(e + kSegLen, ptr[sl + 1]));
        }
      }
      sp.push_back((int)ss.size());
    }
    d->nseg = (int)ss.size();
    if ((rc = upload(&d->seg_slot, ss)) || (rc = upload(&d->seg_rng, rng)) || (rc = upload(&d->seg_ptr, sp))) {
      delete d;
      return rc;
    }
    d->part_rows = ss.size();
  }
  {
    // reverse recursions: segments of every row, the first segment of each level
    std::vector<int> rng, ptr;
    segment_rows(A->bs_ptr, rng, ptr);
    for (size_t lv = 0; lv < T->lvl_ptr.size(); ++lv) d->rs_lvl.push_back(ptr[T->lvl_ptr[lv]]);
    for (size_t lv = 0; lv + 1 < d->rs_lvl.size(); ++lv)
      d->part_rows = std::max(d->part_rows, (size_t)(d->rs_lvl[lv + 1] - d->rs_lvl[lv]));
    if ((rc = upload(&d->rs_rng, rng)) || (rc = upload(&d->rs_ptr, ptr))) { delete d; return rc; }
    std::vector<int> rng2, ptr2;
    segment_rows(A->obs_ptr, rng2, ptr2);
    for (size_t lv = 0; lv < T->olvl_ptr.size(); ++lv) d->ro_lvl.push_back(ptr2[T->olvl_ptr[lv]]);
    for (size_t lv = 0; lv + 1 < d->ro_lvl.size(); ++lv)
      d->part_rows = std::max(d->part_rows, (size_t)(d->ro_lvl[lv + 1] - d->ro_lvl[lv]));
    if ((rc = upload(&d->ro_rng, rng2)) || (rc = upload(&d->ro_ptr, ptr2))) { delete d; return rc; }
    // back-substitution: the bk rows' segments, then the bw rows'
    std::vector<int> brng, kptr, wptr;
    segment_rows(A->bk_ptr, brng, kptr);
    int nk = (int)(brng.size() / 2);
    std::vector<int> wrng;
    segment_rows(A->bw_ptr, wrng, wptr);
    for (int& v : wptr) v += nk;
    brng.insert(brng.end(), wrng.begin(), wrng.end());
    std::vector<int> kind(brng.size() / 2, 0);
    for (size_t g = nk; g < kind.size(); ++g) kind[g] = (int)0x80000000u;
    d->nbseg = (int)kind.size();
    d->part_rows = std::max(d->part_rows, kind.size());
    if ((rc = upload(&d->bseg_kind, kind)) || (rc = upload(&d->bseg_rng, brng)) || (rc = upload(&d->bk_segptr, kptr)) ||
        (rc = upload(&d->bw_segptr, wptr))) {
      delete d;
      return rc;
    }
  }
  if ((rc = upload(&d->bs_ptr, A->bs_ptr)) || (rc = upload(&d->bs_ent, A->bs_ent)) ||
      (rc = upload(&d->bl_ptr, A->bl_ptr)) || (rc = upload(&d->bl_ent, A->bl_ent)) ||
      (rc = upload(&d->obs_ptr, A->obs_ptr)) || (rc = upload(&d->obs_ent, A->obs_ent)) ||
      (rc = upload(&d->obl_ptr, A->obl_ptr)) || (rc = upload(&d->obl_ent, A->obl_ent)) ||
      (rc = upload(&d->hs_ptr, A->hs_ptr)) || (rc = upload(&d->hs_ent, A->hs_ent)) ||
      (rc = upload(&d->hk_ptr, A->hk_ptr)) || (rc = upload(&d->hk_ent, A->hk_ent)) ||
      (rc = upload(&d->dk_ptr, A->dk_ptr)) || (rc = upload(&d->dk_out, A->dk_out)) ||
      (rc = upload(&d->dk_c, A->dk_c)) || (rc = upload(&d->e0_by_key, A->e0_by_key)) ||
      (rc = upload(&d->bk_ptr, A->bk_ptr)) || (rc = upload(&d->bk_ent, A->bk_ent)) ||
      (rc = upload(&d->bw_ptr, A->bw_ptr)) || (rc = upload(&d->bw_ent, A->bw_ent)) ||
      (rc = upload(&d->out_of_state, A->out_of_state))) {
    delete d;
    return rc;
  }
  a->tabs[key] = d;
  *out = d;
  return 0;
}

// reverse pass of one chunk (J subsets per lane); the forward quantities
// (psi, psi_minus, phi, tl, vl, E_0) are in the Ctx buffers
template <int J>
int adjoint_local(Ctx* c, AdjCtx* a, DevTables* T, DevAdj* D, int P, int p0, int nsub, int k, bool keys,
                  cudaStream_t s) {
  const double* psi = (const double*)c->psi;
  const double* pm = (const double*)c->psim;
  const double* phi = (const double*)c->phi;
  const double* tl = (const double*)c->tl;
  const double* vl = (const double*)c->vl;
  const double nv = std::min(P, nsub - p0);
  unsigned gy = (unsigned)(P / (32 * J));
  k_adj_bsub_part<J><<<dim3((unsigned)((D->nbseg + 7) / 8), gy), 256, 0, s>>>(
      P, D->nbseg, D->bseg_kind, D->bseg_rng, D->bk_ent, D->bw_ent, a->wl, pm, phi, a->part);
  size_t no = (size_t)T->nout * P;
  k_adj_bsub_sum<<<(unsigned)((no + 255) / 256), 256, 0, s>>>(P, T->nout, D->bk_segptr, D->bw_segptr, a->part, a->wl,
                                                                a->phib, a->pmb);
  c->n_launches += 2;
  for (int lv = (int)T->olvl_ptr.size() - 2; lv >= 1; --lv) {
    int s0 = T->olvl_ptr[lv], s1 = T->olvl_ptr[lv + 1];
    int g0 = D->ro_lvl[lv], g1 = D->ro_lvl[lv + 1];
    if (s1 <= s0 || g1 <= g0) continue;
    k_rev_part<J><<<dim3((unsigned)((g1 - g0 + 7) / 8), gy), 256, 0, s>>>(P, g0, g1, D->ro_rng, D->obs_ent, tl,
                                                                         a->pmb, a->part);
    size_t nr = (size_t)(s1 - s0) * P;
    k_rev_sum<<<(unsigned)((nr + 255) / 256), 256, 0, s>>>(P, s0, s1, T->olvl_order, D->ro_ptr, g0, a->part, -1.0,
                                                           a->pmb);
    c->n_launches += 2;
  }
  g_prof.done("ph::adjoint: back-substitution, exp(-T) reverse levels", s);
  dim3 gs((unsigned)((T->nstate + 7) / 8), gy);
  k_adj_rows<J><<<gs, 256, 0, s>>>(P, T->nstate, D->hs_ptr, D->hs_ent, D->out_of_state, T->d_ptr, T->d_key, T->d_c,
                                   c->e0loc, vl, a->phib, a->psib);
  c->n_launches++;
  g_prof.done("ph::adjoint: Hamiltonian rows by state (k_adj_rows)", s);
  for (int lv = (int)T->lvl_ptr.size() - 2; lv >= 1; --lv) {
    int s0 = T->lvl_ptr[lv], s1 = T->lvl_ptr[lv + 1];
    int g0 = D->rs_lvl[lv], g1 = D->rs_lvl[lv + 1];
    if (s1 <= s0 || g1 <= g0) continue;
    k_rev_part<J><<<dim3((unsigned)((g1 - g0 + 7) / 8), gy), 256, 0, s>>>(P, g0, g1, D->rs_rng, D->bs_ent, tl,
                                                                         a->psib, a->part);
    size_t nr = (size_t)(s1 - s0) * P;
    k_rev_sum<<<(unsigned)((nr + 255) / 256), 256, 0, s>>>(P, s0, s1, nullptr, D->rs_ptr, g0, a->part, 1.0, a->psib);
    c->n_launches += 2;
  }
  g_prof.done("ph::adjoint: exp(T) reverse levels (k_rev_part, k_rev_sum)", s);
  dim3 gt((unsigned)((D->nseg + 7) / 8), gy);
  k_adj_tbar_part<J><<<gt, 256, 0, s>>>(P, D->nseg, D->seg_slot, D->seg_rng, D->obl_ent, D->bl_ent, pm, a->pmb,
                                        psi, a->psib, a->part);
  size_t ns = (size_t)T->nslot * P;
  k_adj_tbar_sum<<<(unsigned)((ns + 255) / 256), 256, 0, s>>>(P, p0, nsub, T->nslot, D->seg_ptr, a->part,
                                                                a->Tloc[k]);
  c->n_launches += 2;
  g_prof.done("ph::adjoint: amplitude adjoints by slot (k_adj_tbar_part, k_adj_tbar_sum)", s,
              D->nent * 8.0 + 3.0 * D->nent * 8.0 * nv, 2.0 * D->nent * nv);
  if (keys) {
    k_adj_S<<<(unsigned)(P / 32), 256, 0, s>>>(P, T->nout, T->out_state, psi, a->phib, a->S);
    dim3 gk((unsigned)((T->nkey + 7) / 8), gy);
    k_adj_vbar<J><<<gk, 256, 0, s>>>(P, p0, nsub, T->nkey, D->hk_ptr, D->hk_ent, D->dk_ptr, D->dk_out, D->dk_c,
                                     D->e0_by_key, T->out_state, psi, a->phib, a->S, a->Vloc[k]);
    c->n_launches += 2;
    g_prof.done("ph::adjoint: integral-key adjoints (k_adj_S, k_adj_vbar)", s);
  }
  CK(cudaGetLastError());
  return 0;
}

// grad_t L at amplitudes c->t and multipliers lam (layout, copies consistent)
// into grad (unique slots assembled, copies filled); with keys also the
// adjoints of the gathered integrals into a->Gb[m] (label sets in colex order)
//
// cache: keep (or reuse) the forward quantities of every chunk in HBM; the
// caller guarantees that t is unchanged while a->fwd_valid is set
int adjoint_pass(Ctx* c, AdjCtx* a, int N, int K, int KH, const double* lam, double* grad, bool keys,
                 cudaStream_t s, bool cache = false) {
  int rc;
  int kfull = K + KH, kmax = std::min(kfull, N);
  const int key = (N * 8 + K) * 8 + KH;
  bool reuse = cache && a->fwd_valid && a->fwd_key == key;
  bool fill = cache && !reuse;
  if (fill) {
    // the cache grows only while it stays within half of the free device memory
    size_t extra = 0;
    for (int k = 1; k <= kmax; ++k) {
      DevTables* T;
      if ((rc = dev_tables(c, k, K, KH, &T))) return rc;
      int nsub = c->nsub[k];
      int J = nsub >= 384 ? 4 : nsub >= 96 ? 2 : 1;
      int P = chunk_size(nsub, T->nstate, 2 * sizeof(double), 32 * J);
      size_t need = fwd_chunk_bytes(T, P) * (size_t)((nsub + P - 1) / P);
      if (need > a->fwd_cap[k]) extra += need;
    }
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    if (extra > fr / 2) fill = false;
    a->fwd_valid = false;
  }

  AsmArgs A{};
  A.kmax = kmax;
  KeyAsm KA{};
  KA.kmax = kmax;
  const double* t = c->t;
  for (int k = 1; k <= kmax; ++k) {
    double ck = moebius(N, k, kfull), ce = k <= KH ? moebius(N, k, KH) : 0.0;
    if (ck == 0.0 && ce == 0.0) continue;
    DevTables* T;
    DevAdj* D;
    if ((rc = dev_tables(c, k, K, KH, &T)) || (rc = dev_adjoint(a, k, K, KH, &D))) return rc;
    int nsub = c->nsub[k];
    int J = nsub >= 384 ? 4 : nsub >= 96 ? 2 : 1;
    int P = chunk_size(nsub, T->nstate, 2 * sizeof(double), 32 * J);  // psi and psibar
    size_t pd = (size_t)P * sizeof(double);
    if ((rc = grow_buf(&c->psi, &c->cap_psi, T->nstate * pd)) || (rc = grow_buf(&c->psim, &c->cap_out, T->nout * pd)) ||
        (rc = grow_buf(&c->phi, &c->cap_phi, T->nout * pd)) || (rc = grow_buf(&c->tl, &c->cap_tl, T->nslot * pd)) ||
        (rc = grow_buf(&c->vl, &c->cap_vl, T->nkey * pd)) || (rc = grow_buf((void**)&c->e0loc, &c->cap_e0, pd)) ||
        (rc = grow_buf((void**)&a->wl, &a->cap_w, T->nout * pd)) ||
        (rc = grow_buf((void**)&a->phib, &a->cap_phib, T->nout * pd)) ||
        (rc = grow_buf((void**)&a->pmb, &a->cap_pmb, T->nout * pd)) ||
        (rc = grow_buf((void**)&a->psib, &a->cap_psib, T->nstate * pd)) ||
        (rc = grow_buf((void**)&a->S, &a->cap_S, pd)) ||
        (rc = grow_buf((void**)&a->part, &a->cap_part, D->part_rows * pd)) ||
        (rc = grow_buf((void**)&a->Tloc[k], &a->cap_T[k], (size_t)(T->nslot + 1) * nsub * sizeof(double))))
      return rc;
    if (keys && (rc = grow_buf((void**)&a->Vloc[k], &a->cap_V[k], (size_t)T->nkey * nsub * sizeof(double))))
      return rc;
    const size_t cb = fwd_chunk_bytes(T, P);
    if (fill && (rc = grow_buf(&a->fwd[k], &a->fwd_cap[k], cb * (size_t)((nsub + P - 1) / P)))) return rc;
    for (int p0 = 0; p0 < nsub; p0 += P) {
      // the working buffers as grown above, put back after the chunk
      struct Saved { void *psi, *psim, *phi, *tl, *vl; double* e0; } saved{c->psi, c->psim, c->phi, c->tl, c->vl,
                                                                          c->e0loc};
      if (fill || reuse) {
        // this chunk's forward quantities live in the cache
        double* base = (double*)((char*)a->fwd[k] + cb * (size_t)(p0 / P));
        c->psi = base;
        c->psim = base + (size_t)T->nstate * P;
        c->phi = base + (size_t)(T->nstate + T->nout) * P;
        c->tl = base + (size_t)(T->nstate + 2 * (size_t)T->nout) * P;
        c->vl = base + (size_t)(T->nstate + 2 * (size_t)T->nout + T->nslot) * P;
        c->e0loc = base + (size_t)(T->nstate + 2 * (size_t)T->nout + T->nslot + T->nkey) * P;
      }
      double* tl = (double*)c->tl;
      double* vl = (double*)c->vl;
      size_t nt = (size_t)T->nslot * P, nk = (size_t)T->nkey * P, nw = (size_t)(T->nslot + 1) * P;
      if (!reuse) {
        k_gather_amp<double><<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(P, p0, nsub, k, T->nslot, T->slot_desc,
                                                                          c->subs[k], N, t, tl);
        k_gather_int<double><<<(unsigned)((nk + 255) / 256), 256, 0, s>>>(P, p0, nsub, k, T->nkey, T->key_desc,
                                                                          c->subs[k], N, c->G1, c->G2, c->G3, c->G4,
                                                                          vl);
        k_set_ref<double><<<(P + 127) / 128, 128, 0, s>>>(P, (double*)c->psi, (double*)c->psim, T->ne0, T->e0_key,
                                                          T->e0_cd, vl, c->e0loc);
        c->n_launches += 3;
      }
      k_gather_w<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(P, p0, nsub, k, T->nslot, T->slot_desc, c->subs[k], N,
                                                              lam, ck, ce, a->wl);
      c->n_launches++;
      g_prof.done("ph::gather (amplitudes, integrals, multipliers)", s,
                  (double)((reuse ? 1 : 2) * T->nslot + (reuse ? 0 : T->nkey)) * P * 16.0);
      if (!reuse) {
        if (J == 4) rc = local_problem<double, 4>(c, T, P, p0, nsub, k, s, false);
        else if (J == 2) rc = local_problem<double, 2>(c, T, P, p0, nsub, k, s, false);
        else rc = local_problem<double, 1>(c, T, P, p0, nsub, k, s, false);
      }
      if (!rc) {
        if (J == 4) rc = adjoint_local<4>(c, a, T, D, P, p0, nsub, k, keys, s);
        else if (J == 2) rc = adjoint_local<2>(c, a, T, D, P, p0, nsub, k, keys, s);
        else rc = adjoint_local<1>(c, a, T, D, P, p0, nsub, k, keys, s);
      }
      c->psi = saved.psi; c->psim = saved.psim; c->phi = saved.phi; c->tl = saved.tl; c->vl = saved.vl;
      c->e0loc = saved.e0;
      if (rc) return rc;
    }
    A.Rloc[k] = a->Tloc[k]; A.nout[k] = T->nslot + 1; A.nsub[k] = nsub; A.c[k] = 1.0;
    KA.V[k] = a->Vloc[k]; KA.nkey[k] = T->nkey; KA.nsub[k] = nsub;
  }
  size_t L = layout_len(N, K);
  CK(cudaMemsetAsync(grad, 0, sizeof(double) * L, s));
  const int nch[4] = {0, 3, 29, kNA3};
  for (int m = 1; m <= std::min(K, N); ++m) {
    size_t nt = (size_t)c->nsub[m] * nch[m];
    k_assemble<<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(N, m, nch[m], c->subs[m], c->nsub[m], A, grad);
    c->n_launches++;
  }
  k_fill_copies<<<(unsigned)((L + 255) / 256), 256, 0, s>>>(L, N, K, grad);
  c->n_launches++;
  if (keys) {
    const int nk[5] = {0, 20, 232, 576, 384};
    for (int m = 1; m <= std::min(std::min(KH, 4), N); ++m) {
      size_t nt = (size_t)c->nsub[m] * nk[m];
      if ((rc = grow_buf((void**)&a->Gb[m], &a->cap_G[m], nt * sizeof(double)))) return rc;
      k_assemble_keys<<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(N, m, c->subs[m], c->nsub[m], KA, a->Gb[m]);
      c->n_launches++;
    }
  }
  g_prof.done("ph::assembly of the adjoints", s);
  CK(cudaGetLastError());
  if (fill) {
    a->fwd_valid = true;
    a->fwd_key = key;
  }
  return 0;
}

int grow_adjoint_state(AdjCtx* a, size_t L) {
  if (L <= a->cap_L) return 0;
  if (a->lam) cudaFree(a->lam);
  if (a->grad) cudaFree(a->grad);
  a->lam = a->grad = nullptr;
  a->cap_L = 0;
  CK(cudaMalloc((void**)&a->lam, sizeof(double) * L));
  CK(cudaMalloc((void**)&a->grad, sizeof(double) * L));
  a->cap_L = L;
  return 0;
}

// Lambda equations at the amplitudes in c->t: grad_t L(t, lambda) = 0 by
// Jacobi steps lambda += grad / D with device DIIS (FP64), from lambda = 0
int solve_lambda(Ctx* c, AdjCtx* a, Workspace* w, int N, int K, int KH, const ppq_opts& o, cudaStream_t s,
                 double* res_out, int* iters_out) {
  int rc;
  size_t L = layout_len(N, K);
  if ((rc = grow_adjoint_state(a, L))) return rc;
  CK(cudaMemsetAsync(a->lam, 0, sizeof(double) * L, s));
  a->fwd_valid = false;  // new amplitudes: the first reverse pass refills the cache
  PhSolver S(c, w, N, K, KH, o, s);
  if ((rc = S.init())) return rc;
  std::vector<int> ring;
  double res = 0.0;
  int it = 1, status = 1;
  for (; it <= o.max_iter; ++it) {
    if ((rc = adjoint_pass(c, a, N, K, KH, a->lam, a->grad, false, s, true))) return rc;
    if ((rc = S.norm(a->grad, &res))) return rc;
    if (trace_on()) fprintf(stderr, "ph lambda %3d |grad_t L| %.3e\n", it, res);
    if (!isfinite(res) || res > 1e6) { status = 2; break; }
    if (res <= o.r_tol) { status = 0; break; }
    if ((rc = S.step_on(a->lam, a->grad, it, ring))) return rc;
    k_fill_copies<<<(unsigned)((L + 255) / 256), 256, 0, s>>>(L, N, K, a->lam);
    c->n_launches++;
  }
  *res_out = res;
  *iters_out = std::min(it, o.max_iter);
  return status;
}

// dE_total/dh, dE_total/d(pq|rs) (both symmetrised) and dE/dkappa at the
// amplitudes in c->t and multipliers in a->lam
int integral_gradients(Ctx* c, AdjCtx* a, Workspace* w, const Problem& P, int K, int KH, cudaStream_t s) {
  int rc;
  int N = P.N, n = P.n;
  size_t n2 = (size_t)n * n, n4 = n2 * n2;
  if (a->cap_n < (size_t)n) {
    double** ps[] = {&a->dhp, &a->gh_raw, &a->gh, &a->gv_raw, &a->gv, &a->dk, &a->ab};
    for (double** p : ps)
      if (*p) { cudaFree(*p); *p = nullptr; }
    a->cap_n = 0;
    CK(cudaMalloc((void**)&a->dhp, sizeof(double) * n2));
    CK(cudaMalloc((void**)&a->gh_raw, sizeof(double) * n2));
    CK(cudaMalloc((void**)&a->gh, sizeof(double) * n2));
    CK(cudaMalloc((void**)&a->gv_raw, sizeof(double) * n4));
    CK(cudaMalloc((void**)&a->gv, sizeof(double) * n4));
    CK(cudaMalloc((void**)&a->dk, sizeof(double) * n2));
    CK(cudaMalloc((void**)&a->ab, sizeof(double) * 2 * n2));
    a->cap_n = n;
  }
  if ((rc = adjoint_pass(c, a, N, K, KH, a->lam, a->grad, true, s, true))) return rc;
  a->fwd_valid = false;
  CK(cudaMemsetAsync(a->dhp, 0, sizeof(double) * n2, s));
  CK(cudaMemsetAsync(a->gv_raw, 0, sizeof(double) * n4, s));
  const int nk[5] = {0, 20, 232, 576, 384};
  for (int m = 1; m <= std::min(std::min(KH, 4), N); ++m) {
    size_t nt = (size_t)c->nsub[m] * nk[m];
    k_scatter_keys<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(n, m, c->subs[m], c->nsub[m], a->Gb[m], w->occ,
                                                                w->vir, a->dhp, a->gv_raw);
    c->n_launches++;
  }
  // h' = h for K_H >= 3 (no (pq|ii) is truncated); for K_H = 2 the chain rule
  // through h' = f - sum_i [2 v'(pq|ii) - v'(pi|iq)]; E_ref in both
  ppq::adj::k_grad_chain<<<(unsigned)((n2 + 127) / 128), 128, 0, s>>>(n, N, a->dhp, w->occ, w->lab, a->gh_raw,
                                                                      a->gv_raw, KH == 2 ? 1 : 0);
  ppq::adj::k_sym_h<<<(unsigned)((n2 + 127) / 128), 128, 0, s>>>(n, a->gh_raw, a->gh);
  ppq::adj::k_sym_v<<<(unsigned)((n4 + 255) / 256), 256, 0, s>>>(n, a->gv_raw, a->gv);
  ppq::adj::k_orbital_grad<<<(unsigned)((n2 + 127) / 128), 128, 0, s>>>(n, P.h, P.eri, a->gh, a->gv, a->ab);
  ppq::adj::k_orbital_final<<<(unsigned)((n2 + 127) / 128), 128, 0, s>>>(n, a->ab, a->dk);
  c->n_launches += 5;
  g_prof.done("ph::integral and orbital gradients", s);
  CK(cudaGetLastError());
  return 0;
}

}  // namespace ph

extern "C" {

int ph_lagrangian_gradient(int n_pairs, const int* occ_of_pair, const int* vir_of_pair, const double* h,
                           const double* eri, const double* t, const double* lam, int K_H, double* grad,
                           double* e_corr, void* stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_err.clear();
  cudaStream_t s = (cudaStream_t)stream;
  int KH = K_H == 0 ? 3 : K_H;
  if (KH != 2 && KH != 3) return fail(-4, "ph_lagrangian_gradient: K_H must be 0 (= 3), 2 or 3");
  if (!t || !lam || !grad) return fail(-2, "t, lam and grad must be non-null");
  if (n_pairs > 127) return fail(-1, "n_pairs must be <= 127 for the label-subset residual");
  Workspace* w = nullptr;
  Problem P;
  int rc = prepare(n_pairs, occ_of_pair, vir_of_pair, h, eri, 1, s, &w, &P);
  if (rc) return rc;
  ph::Ctx* c = ph::ctx();
  ph::AdjCtx* a = ph::adj_ctx();
  if ((rc = ph::stage_ph(c, w, P, KH, s))) return rc;
  int N = n_pairs, K = 3;
  size_t L = ph::layout_len(N, K);
  if ((rc = ph::grow_solver(c, L, 1)) || (rc = ph::grow_adjoint_state(a, L))) return rc;
  unsigned lb = (unsigned)((L + 255) / 256);
  CK(cudaMemcpyAsync(c->t, t, sizeof(double) * L, cudaMemcpyDefault, s));
  CK(cudaMemcpyAsync(a->lam, lam, sizeof(double) * L, cudaMemcpyDefault, s));
  ph::k_fill_copies<<<lb, 256, 0, s>>>(L, N, K, c->t);
  ph::k_fill_copies<<<lb, 256, 0, s>>>(L, N, K, a->lam);
  if (e_corr && (rc = ph::residual_any(c, N, K, KH, 0, c->t, c->r, c->e, s))) return rc;
  if ((rc = ph::adjoint_pass(c, a, N, K, KH, a->lam, a->grad, false, s))) return rc;
  CK(cudaMemcpyAsync(grad, a->grad, sizeof(double) * L, cudaMemcpyDefault, s));
  if (e_corr) CK(cudaMemcpyAsync(c->host, c->e, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (e_corr) *e_corr = c->host[0];
  return 0;
}

int ph_gradient(int n_pairs, const int* occ_of_pair, const int* vir_of_pair, const double* h, const double* eri,
                double e_const, const ppq_opts* opts, double* t_out, double* lam_out, double* dE_dh,
                double* dE_deri, double* dE_dkappa, double* e_total, ppq_info* info, void* stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_err.clear();
  auto wall0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  ppq_opts o;
  if (opts) o = *opts; else ppq_default_opts(&o);
  int KH = o.K_H == 0 ? 3 : o.K_H;
  if (KH != 2 && KH != 3) return fail(-4, "ph_gradient: K_H must be 0 (= 3), 2 or 3");
  if (o.guess != 0) return fail(-4, "ph_gradient starts from zero amplitudes (guess = 0)");
  if (!eri) return fail(-2, "eri must be non-null");
  double ec = 0.0, et = 0.0;
  ppq_info si;
  int status = subset_solve(3, KH, n_pairs, occ_of_pair, vir_of_pair, h, eri, nullptr, 0, e_const, o, nullptr,
                            nullptr, &ec, &et, &si, s, wall0);
  if (status < 0) return status;
  Workspace* w = nullptr;
  Problem P;
  int rc = prepare(n_pairs, occ_of_pair, vir_of_pair, h, eri, 1, s, &w, &P);
  if (rc) return rc;
  // the kernel profile of the amplitude solve continues through the reverse passes
  if (o.profile) {
    g_prof.on = true;
    g_prof.start(s);
  }
  struct ProfOff { ~ProfOff() { g_prof.on = false; } } prof_off;
  ph::Ctx* c = ph::ctx();
  ph::AdjCtx* a = ph::adj_ctx();
  int N = n_pairs, n = 2 * N, K = 3;
  size_t L = ph::layout_len(N, K), n2 = (size_t)n * n;
  ppq_opts ol = o;
  ol.precision = 0;
  double lres = 0.0;
  int liters = 0;
  int lstat = ph::solve_lambda(c, a, w, N, K, KH, ol, s, &lres, &liters);
  if (lstat < 0) return lstat;
  if ((rc = ph::integral_gradients(c, a, w, P, K, KH, s))) return rc;
  if (t_out) CK(cudaMemcpyAsync(t_out, c->t, sizeof(double) * L, cudaMemcpyDefault, s));
  if (lam_out) CK(cudaMemcpyAsync(lam_out, a->lam, sizeof(double) * L, cudaMemcpyDefault, s));
  if (dE_dh) CK(cudaMemcpyAsync(dE_dh, a->gh, sizeof(double) * n2, cudaMemcpyDefault, s));
  if (dE_deri) CK(cudaMemcpyAsync(dE_deri, a->gv, sizeof(double) * n2 * n2, cudaMemcpyDefault, s));
  if (dE_dkappa) CK(cudaMemcpyAsync(dE_dkappa, a->dk, sizeof(double) * n2, cudaMemcpyDefault, s));
  CK(cudaStreamSynchronize(s));
  if (e_total) *e_total = et;
  if (info) {
    *info = si;
    info->status = std::max(status, lstat);
    info->t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
  }
  return std::max(status, lstat);
}

}  // extern "C"
