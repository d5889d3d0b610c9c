// ph_tables.cuh -- host generator of the structure tables of the label-subset
// expansion (the exact K-pair residual of the Theory section evaluated from
// local problems over at most K + K_H pairing labels).
//
// Sites and monomials.  Each pairing label is a site with four spin orbitals
// (0 = o_up, 1 = o_dn, 2 = v_up, 3 = v_dn) and 16 local states |m> = E^m |ref>,
// m a 4-bit mask, E^m = a+_{v_up}^{b2} a+_{v_dn}^{b3} a_{o_dn}^{b1} a_{o_up}^{b0}
// (bits 0/1 open a hole, bits 2/3 add a particle).  A k-site configuration is
// the 4k-bit code with site j in bits 4j..4j+3, |code> = E_0^{m_0} ... E_{k-1}^{m_{k-1}} |ref>;
// codes of the zero-charge, zero-S_z sector are the "states".  Every sign is
// obtained by applying creation / annihilation operators to Jordan-Wigner
// determinants (4j + l ordering), never by hand.
//
// Amplitude channels (Eq. decompose, Tables I-II): A1 (3 single-site
// monomials), A2 (29 two-site pairs), A3 (303 three-site triples) of nonzero
// monomials with zero total charge and S_z, in the order of the C-ABI layout.
// Integral keys: 20 per site, 232 per two sites, 576 per three sites and 384
// per four (untruncated integrals, K_H = 4 here), the (pq|rs) and one-body
// elements whose orbitals span exactly those sites.
//
// For k sites the generator produces, once per (k, K, K_H):
//   * the sector states, sorted by level (number of hole-particle pairs);
//   * the recursion of psi = exp(T)|ref> over the sector: for a state s with
//     lowest set bit b, psi(s) = sum over clusters c (a channel on <= K sites)
//     with b in c and c inside s of sign(c, s \ c) t_c psi(s \ c), where
//     E^c E^{s\c} = sign E^s (every set of disjoint clusters covering s has
//     exactly one cluster holding b, and exp(T) = prod_c (1 + t_c E^c));
//   * the same recursion over the outputs (states on at most K sites) for
//     exp(-T)|ref>;
//   * the Hamiltonian rows phi_kappa = <kappa| H |psi> for every output kappa:
//     (state s, integral key slot, coefficient) with <kappa|term|s> from JW,
//     the diagonal s = kappa in a list of its own;
//   * the back-substitution R_mu = sum_{kappa subset mu} sign(kappa, mu\kappa)
//     [exp(-T)](mu \ kappa) phi'_kappa, phi' = phi - E_0 psi.
#pragma once
#include <stdint.h>

#include <algorithm>
#include <array>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

namespace ph {

constexpr int kMaxSites = 6;

inline int popc(uint32_t x) { return __builtin_popcount(x); }
inline int binom(int n, int r) {
  if (r < 0 || r > n) return 0;
  long long c = 1;
  for (int i = 1; i <= r; ++i) c = c * (n - r + i) / i;
  return (int)c;
}
// colex rank of a sorted position set (p0 < p1 < ...): sum_i C(p_i, i + 1)
inline int colex_rank(const int* p, int m) {
  int r = 0;
  for (int i = 0; i < m; ++i) r += binom(p[i], i + 1);
  return r;
}

// ------------------------------------------------------------ Jordan-Wigner
// apply a (dag = 1) or a+ ... to a determinant of spin orbitals so = 4 j + l
inline bool jw_apply(uint32_t& det, int so, int dag, int& sg) {
  int on = (det >> so) & 1;
  if (dag == on) return false;
  if (popc(det & ((1u << so) - 1u)) & 1) sg = -sg;
  det ^= 1u << so;
  return true;
}
// E^m on site j (the operators of E^m applied right to left)
inline bool jw_mono(uint32_t& det, int j, int m, int& sg) {
  if ((m & 1) && !jw_apply(det, 4 * j + 0, 0, sg)) return false;
  if ((m & 2) && !jw_apply(det, 4 * j + 1, 0, sg)) return false;
  if ((m & 8) && !jw_apply(det, 4 * j + 3, 1, sg)) return false;
  if ((m & 4) && !jw_apply(det, 4 * j + 2, 1, sg)) return false;
  return true;
}
// E_0^{m_0} ... E_{k-1}^{m_{k-1}} applied to det (site k-1 first)
inline bool jw_code(uint32_t code, int k, uint32_t& det, int& sg) {
  for (int j = k - 1; j >= 0; --j)
    if (!jw_mono(det, j, (code >> (4 * j)) & 15, sg)) return false;
  return true;
}
inline uint32_t ref_det(int k) {
  uint32_t d = 0;
  for (int j = 0; j < k; ++j) d |= 3u << (4 * j);
  return d;
}
// determinant and sign of |code>
inline void state_det(uint32_t code, int k, uint32_t* det, int* sg) {
  uint32_t d = ref_det(k);
  int s = 1;
  bool ok = jw_code(code, k, d, s);
  (void)ok;
  *det = d;
  *sg = s;
}
// the code whose determinant is det (holes where occupied orbitals are empty)
inline uint32_t det_code(uint32_t det, int k) {
  uint32_t c = 0;
  for (int j = 0; j < k; ++j) {
    uint32_t b = (det >> (4 * j)) & 15u;
    c |= (((~b) & 3u) | (b & 12u)) << (4 * j);
  }
  return c;
}
// E^c E^r = sign E^{c|r} (0 if c and r overlap), by JW
inline int merge_sign(uint32_t c, uint32_t r, int k) {
  if (c & r) return 0;
  uint32_t d;
  int sr;
  state_det(r, k, &d, &sr);
  int sc = 1;
  if (!jw_code(c, k, d, sc)) return 0;
  uint32_t d2;
  int s2;
  state_det(c | r, k, &d2, &s2);
  return sr * sc * s2;
}

// ------------------------------------------------------------ site algebra
struct Algebra {
  int qc[16], qs[16];
  std::vector<int> A1;
  std::vector<std::array<int, 2>> A2;
  std::vector<std::array<int, 3>> A3;
  std::vector<std::array<int, 5>> key[5];  // (0 = one-body h', 1 = (pq|rs); local orbitals)
  Algebra() {
    for (int m = 0; m < 16; ++m) {
      qc[m] = popc(m & 12) - popc(m & 3);
      qs[m] = ((m >> 2) & 1) - ((m >> 3) & 1) - ((m & 1) - ((m >> 1) & 1));
    }
    for (int m = 1; m < 16; ++m)
      if (qc[m] == 0 && qs[m] == 0) A1.push_back(m);
    for (int a = 1; a < 16; ++a)
      for (int b = 1; b < 16; ++b)
        if (qc[a] + qc[b] == 0 && qs[a] + qs[b] == 0) A2.push_back({a, b});
    for (int a = 1; a < 16; ++a)
      for (int b = 1; b < 16; ++b)
        for (int c = 1; c < 16; ++c)
          if (qc[a] + qc[b] + qc[c] == 0 && qs[a] + qs[b] + qs[c] == 0) A3.push_back({a, b, c});
    // keys: local spatial orbital o lives on site o / 2 (x = o % 2: 0 occupied, 1 virtual)
    for (int x = 0; x < 2; ++x)
      for (int y = 0; y < 2; ++y) key[1].push_back({0, x, y, 0, 0});
    for (int p = 0; p < 2; ++p)
      for (int q = 0; q < 2; ++q)
        for (int r = 0; r < 2; ++r)
          for (int s = 0; s < 2; ++s) key[1].push_back({1, p, q, r, s});
    for (int p = 0; p < 4; ++p)
      for (int q = 0; q < 4; ++q)
        if (p / 2 != q / 2) key[2].push_back({0, p, q, 0, 0});
    for (int p = 0; p < 4; ++p)
      for (int q = 0; q < 4; ++q)
        for (int r = 0; r < 4; ++r)
          for (int s = 0; s < 4; ++s) {
            int sites = (1 << (p / 2)) | (1 << (q / 2)) | (1 << (r / 2)) | (1 << (s / 2));
            if (popc(sites) == 2) key[2].push_back({1, p, q, r, s});
          }
    for (int p = 0; p < 6; ++p)
      for (int q = 0; q < 6; ++q)
        for (int r = 0; r < 6; ++r)
          for (int s = 0; s < 6; ++s) {
            int sites = (1 << (p / 2)) | (1 << (q / 2)) | (1 << (r / 2)) | (1 << (s / 2));
            if (popc(sites) == 3) key[3].push_back({1, p, q, r, s});
          }
    // four labels (untruncated integrals): every orbital on a different site
    for (int p = 0; p < 8; ++p)
      for (int q = 0; q < 8; ++q)
        for (int r = 0; r < 8; ++r)
          for (int s = 0; s < 8; ++s) {
            int sites = (1 << (p / 2)) | (1 << (q / 2)) | (1 << (r / 2)) | (1 << (s / 2));
            if (popc(sites) == 4) key[4].push_back({1, p, q, r, s});
          }
  }
  int nch(int m) const { return m == 1 ? (int)A1.size() : m == 2 ? (int)A2.size() : (int)A3.size(); }
  int nkey(int m) const { return (int)key[m].size(); }
  // monomial of channel ch of an m-site cluster at its i-th site
  int mono(int m, int ch, int i) const { return m == 1 ? A1[ch] : m == 2 ? A2[ch][i] : A3[ch][i]; }
};

inline const Algebra& algebra() {
  static Algebra a;
  return a;
}

// packed descriptor of (sorted positions, index):
// npos | p0 << 4 | p1 << 8 | p2 << 12 | p3 << 16 | idx << 20
constexpr int kDescIdx = 20;
inline int pack_desc(int m, const int* p, int idx) {
  int d = m;
  for (int i = 0; i < m; ++i) d |= p[i] << (4 + 4 * i);
  return d | (idx << kDescIdx);
}

// position sets of size m (1..4) among k sites, in colex order
inline std::vector<std::array<int, 4>> position_sets(int k, int m) {
  std::vector<std::array<int, 4>> out(binom(k, m));
  std::array<int, 4> p{0, 0, 0, 0};
  for (int i = 0; i < m; ++i) p[i] = i;
  for (;;) {
    out[colex_rank(p.data(), m)] = p;
    int x = m - 1;
    while (x >= 0 && p[x] == k - m + x) --x;
    if (x < 0) break;
    ++p[x];
    for (int y = x + 1; y < m; ++y) p[y] = p[y - 1] + 1;
  }
  return out;
}

// ------------------------------------------------------------ tables of k sites
struct Tables {
  int k = 0, K = 0, KH = 0;
  int nstate = 0, nslot = 0, nout = 0, nkey = 0, nlevel = 0;
  std::vector<uint32_t> code;                  // sector states, by level
  std::vector<int> lvl_ptr;                    // [nlevel + 1]
  std::vector<int> ent_ptr, ent_sub;           // recursion of exp(T)|ref> over the sector
  std::vector<int16_t> ent_slot;               // 2 slot + (sign < 0)
  std::vector<int> slot_desc;                  // clusters: positions and channel
  std::vector<int> out_state;                  // output -> sector state (output 0 = ref)
  std::vector<int> out_desc;                   // outputs: positions and channel
  std::vector<int> olvl_ptr, olvl_order;       // outputs by level
  std::vector<int> oent_ptr, oent_sub;         // recursion over outputs (sub as output index)
  std::vector<int16_t> oent_slot;
  std::vector<int> key_desc;                   // key slots: positions and key
  std::vector<int> h_ptr, h_s;                 // Hamiltonian rows per output, off the diagonal
  std::vector<int16_t> h_key;
  std::vector<double> h_c;
  std::vector<int> d_ptr;                      // diagonal <kappa|H|kappa> per output
  std::vector<int16_t> d_key;
  std::vector<double> d_c;
  std::vector<int16_t> e0_key;                 // <ref| H |ref>
  std::vector<double> e0_c;
  std::vector<int> b_ptr, b_k, b_w;            // back-substitution per output (w: 2 out + sign bit)
  size_t bytes() const {
    return code.size() * 4 + ent_ptr.size() * 4 + ent_sub.size() * 4 + ent_slot.size() * 2 +
           h_s.size() * 4 + h_key.size() * 2 + h_c.size() * 8 + d_key.size() * 10 + b_k.size() * 8;
  }
};

inline int build_tables(int k, int K, int KH, Tables* T, int nthreads = 0) {
  const Algebra& A = algebra();
  if (k < 1 || k > kMaxSites || K < 1 || K > 3 || KH < 1 || KH > 4) return -1;
  T->k = k; T->K = K; T->KH = KH;
  // ---- sector states sorted by level then code
  const uint32_t ncode = 1u << (4 * k);
  std::vector<int> index(ncode, -1);
  std::vector<std::vector<uint32_t>> bylvl(2 * k + 1);
  for (uint32_t c = 0; c < ncode; ++c) {
    int q = 0, s = 0;
    for (int j = 0; j < k; ++j) {
      int m = (c >> (4 * j)) & 15;
      q += A.qc[m]; s += A.qs[m];
    }
    if (q == 0 && s == 0) bylvl[popc(c) / 2].push_back(c);
  }
  T->nlevel = 2 * k + 1;
  T->lvl_ptr.assign(1, 0);
  for (auto& v : bylvl) {
    for (uint32_t c : v) {
      index[c] = (int)T->code.size();
      T->code.push_back(c);
    }
    T->lvl_ptr.push_back((int)T->code.size());
  }
  T->nstate = (int)T->code.size();
  // ---- clusters (slots): sites in colex order of their position sets
  struct Cl { uint32_t code; int slot; };
  std::vector<std::vector<Cl>> bucket(4 * k);  // by lowest bit
  int slot = 0;
  for (int m = 1; m <= std::min(K, k); ++m) {
    auto sets = position_sets(k, m);
    for (size_t si = 0; si < sets.size(); ++si)
      for (int ch = 0; ch < A.nch(m); ++ch) {
        uint32_t c = 0;
        for (int i = 0; i < m; ++i) c |= (uint32_t)A.mono(m, ch, i) << (4 * sets[si][i]);
        bucket[__builtin_ctz(c)].push_back({c, slot});
        T->slot_desc.push_back(pack_desc(m, sets[si].data(), ch));
        ++slot;
      }
  }
  T->nslot = slot;
  // ---- recursion over the sector
  std::vector<std::vector<int>> es(T->nstate), eslot(T->nstate);
  int nth = nthreads > 0 ? nthreads : (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  auto rec_worker = [&](int t0) {
    for (int si = 1 + t0; si < T->nstate; si += nth) {
      uint32_t s = T->code[si];
      int b = __builtin_ctz(s);
      for (const Cl& cl : bucket[b]) {
        if (cl.code & ~s) continue;
        uint32_t r = s & ~cl.code;
        int sg = merge_sign(cl.code, r, k);
        if (!sg || index[r] < 0) continue;
        es[si].push_back(index[r]);
        eslot[si].push_back(2 * cl.slot + (sg < 0 ? 1 : 0));
      }
    }
  };
  {
    std::vector<std::thread> th;
    for (int t = 0; t < nth; ++t) th.emplace_back(rec_worker, t);
    for (auto& x : th) x.join();
  }
  T->ent_ptr.assign(1, 0);
  for (int si = 0; si < T->nstate; ++si) {
    T->ent_sub.insert(T->ent_sub.end(), es[si].begin(), es[si].end());
    for (int v : eslot[si]) T->ent_slot.push_back((int16_t)v);
    T->ent_ptr.push_back((int)T->ent_sub.size());
    std::vector<int>().swap(es[si]);
    std::vector<int>().swap(eslot[si]);
  }
  // ---- outputs: reference, then states on m = 1..K sites (colex sets, channel order)
  std::vector<int> out_of_state(T->nstate, -1);
  T->out_state.push_back(index[0]);
  T->out_desc.push_back(0);
  out_of_state[index[0]] = 0;
  for (int m = 1; m <= std::min(K, k); ++m) {
    auto sets = position_sets(k, m);
    for (size_t si = 0; si < sets.size(); ++si)
      for (int ch = 0; ch < A.nch(m); ++ch) {
        uint32_t c = 0;
        for (int i = 0; i < m; ++i) c |= (uint32_t)A.mono(m, ch, i) << (4 * sets[si][i]);
        int st = index[c];
        if (st < 0) return -2;
        out_of_state[st] = (int)T->out_state.size();
        T->out_state.push_back(st);
        T->out_desc.push_back(pack_desc(m, sets[si].data(), ch));
      }
  }
  T->nout = (int)T->out_state.size();
  // outputs by level, recursion over outputs (exp(-T) on the outputs)
  {
    std::vector<std::vector<int>> ol(2 * k + 1);
    for (int o = 0; o < T->nout; ++o) ol[popc(T->code[T->out_state[o]]) / 2].push_back(o);
    T->olvl_ptr.assign(1, 0);
    for (auto& v : ol) {
      T->olvl_order.insert(T->olvl_order.end(), v.begin(), v.end());
      T->olvl_ptr.push_back((int)T->olvl_order.size());
    }
    T->oent_ptr.assign(1, 0);
    for (int o : T->olvl_order) {
      int st = T->out_state[o];
      for (int e = T->ent_ptr[st]; e < T->ent_ptr[st + 1]; ++e) {
        int so = out_of_state[T->ent_sub[e]];
        if (so < 0) return -3;  // a sub-state of an output is an output
        T->oent_sub.push_back(so);
        T->oent_slot.push_back(T->ent_slot[e]);
      }
      T->oent_ptr.push_back((int)T->oent_sub.size());
    }
  }
  // ---- integral key slots and Hamiltonian rows
  struct Term { int key; double coef; int nop; int so[4]; int dag[4]; };  // ops left to right
  std::vector<Term> terms;
  for (int m = 1; m <= std::min(KH, k); ++m) {
    auto sets = position_sets(k, m);
    for (size_t si = 0; si < sets.size(); ++si)
      for (int j = 0; j < A.nkey(m); ++j) {
        const auto& ky = A.key[m][j];
        int ks = (int)T->key_desc.size();
        T->key_desc.push_back(pack_desc(m, sets[si].data(), j));
        auto so = [&](int o, int sig) { return 4 * sets[si][o / 2] + 2 * (o % 2) + sig; };
        if (ky[0] == 0) {
          for (int s = 0; s < 2; ++s)
            terms.push_back({ks, 1.0, 2, {so(ky[1], s), so(ky[2], s), 0, 0}, {1, 0, 0, 0}});
        } else {
          for (int s1 = 0; s1 < 2; ++s1)
            for (int s2 = 0; s2 < 2; ++s2)
              terms.push_back({ks, 0.5, 4, {so(ky[1], s1), so(ky[3], s2), so(ky[4], s2), so(ky[2], s1)},
                               {1, 1, 0, 0}});
        }
      }
  }
  T->nkey = (int)T->key_desc.size();
  std::vector<std::vector<std::pair<long long, double>>> hrow(T->nout);
  auto h_worker = [&](int t0) {
    for (int o = t0; o < T->nout; o += nth) {
      uint32_t kc = T->code[T->out_state[o]];
      uint32_t kd;
      int ks;
      state_det(kc, k, &kd, &ks);
      auto& row = hrow[o];
      for (const Term& tm : terms) {
        // <kappa| op |s> = <s| op^dagger |kappa>: apply op^dagger (reversed, daggers flipped)
        uint32_t d = kd;
        int sg = ks;
        bool ok = true;
        for (int i = 0; i < tm.nop && ok; ++i) ok = jw_apply(d, tm.so[i], 1 - tm.dag[i], sg);
        if (!ok) continue;
        uint32_t sc = det_code(d, k);
        int st = index[sc];
        if (st < 0) continue;
        uint32_t d2;
        int s2;
        state_det(sc, k, &d2, &s2);
        row.push_back({(long long)st * 65536 + tm.key, tm.coef * sg * s2});
      }
      std::sort(row.begin(), row.end());
      std::vector<std::pair<long long, double>> mg;
      for (auto& e : row) {
        if (!mg.empty() && mg.back().first == e.first) mg.back().second += e.second;
        else mg.push_back(e);
      }
      row.clear();
      for (auto& e : mg)
        if (e.second != 0.0) row.push_back(e);
    }
  };
  {
    std::vector<std::thread> th;
    for (int t = 0; t < nth; ++t) th.emplace_back(h_worker, t);
    for (auto& x : th) x.join();
  }
  // the diagonal is kept apart: <kappa|H|kappa> - E_0 cancels to an
  // excitation energy, which the kernels form from the same integrals in FP64
  T->h_ptr.assign(1, 0);
  T->d_ptr.assign(1, 0);
  for (int o = 0; o < T->nout; ++o) {
    for (auto& e : hrow[o]) {
      int st = (int)(e.first / 65536);
      int16_t ky = (int16_t)(e.first % 65536);
      if (st == T->out_state[o]) {
        T->d_key.push_back(ky);
        T->d_c.push_back(e.second);
        if (o == 0) {
          T->e0_key.push_back(ky);
          T->e0_c.push_back(e.second);
        }
      } else {
        T->h_s.push_back(st);
        T->h_key.push_back(ky);
        T->h_c.push_back(e.second);
      }
    }
    T->h_ptr.push_back((int)T->h_s.size());
    T->d_ptr.push_back((int)T->d_key.size());
  }
  // ---- back-substitution over sub-states of each output
  T->b_ptr.assign(1, 0);
  for (int o = 0; o < T->nout; ++o) {
    uint32_t mu = T->code[T->out_state[o]];
    // every submask kappa of mu (including 0 and mu) that is a sector state
    uint32_t sub = mu;
    for (;;) {
      int st = index[sub];
      if (st >= 0) {
        uint32_t w = mu & ~sub;
        int sw = index[w];
        int ko = out_of_state[st], wo = sw >= 0 ? out_of_state[sw] : -1;
        if (ko < 0 || wo < 0) return -4;
        int sg = merge_sign(sub, w, k);
        if (!sg) return -5;
        T->b_k.push_back(ko);
        T->b_w.push_back(2 * wo + (sg < 0 ? 1 : 0));
      }
      if (sub == 0) break;
      sub = (sub - 1) & mu;
    }
    T->b_ptr.push_back((int)T->b_k.size());
  }
  return 0;
}

// cache of host tables per (k, K, K_H)
inline const Tables* host_tables(int k, int K, int KH, int* rc) {
  static std::mutex mu;
  static std::unique_ptr<Tables> cache[kMaxSites + 1][4][5];
  std::lock_guard<std::mutex> lk(mu);
  *rc = 0;
  if (k < 1 || k > kMaxSites || K < 1 || K > 3 || KH < 1 || KH > 4) {
    *rc = -1;
    return nullptr;
  }
  auto& slot = cache[k][K][KH];
  if (!slot) {
    std::unique_ptr<Tables> T(new Tables());
    *rc = build_tables(k, K, KH, T.get());
    if (*rc) return nullptr;
    slot = std::move(T);
  }
  return slot.get();
}

}  // namespace ph

namespace ph {

// ------------------------------------------------------------ adjoint tables
// The transposed forms of the tables, for the reverse pass of a local problem
// (the Lambda equations and the energy gradient): every entry of the forward
// tables appears once, grouped by the operand it is differentiated against.
struct AdjTables {
  // sector recursion psi(s) = sum sign t_c psi(sub): by sub -> (s, 2 slot + sign);
  // by slot -> (s, sub, sign) packed s | sub << 20 | sign << 40
  std::vector<int> bs_ptr;
  std::vector<unsigned long long> bs_ent;
  std::vector<int> bl_ptr;
  std::vector<unsigned long long> bl_ent;
  // the same for the output recursion (indices are output indices; bs grouped
  // by output, in the level order of the outputs)
  std::vector<int> obs_ptr;
  std::vector<unsigned long long> obs_ent;
  std::vector<int> obl_ptr;
  std::vector<unsigned long long> obl_ent;
  // Hamiltonian rows off the diagonal, by state s -> (kappa, key, coef) and by
  // key -> (kappa, s, coef); coef in {+-1/2, +-1}: kappa | key << 13 |
  // neg << 28 | half << 29 (by state), kappa | s << 13 | neg << 33 | half << 34 (by key)
  std::vector<int> hs_ptr;
  std::vector<unsigned> hs_ent;
  std::vector<int> hk_ptr;
  std::vector<unsigned long long> hk_ent;
  // diagonal entries by key -> (kappa, d_c); E_0 coefficient by key
  std::vector<int> dk_ptr, dk_out;
  std::vector<double> dk_c, e0_by_key;
  // back-substitution by kappa -> (o, w, sign) and by w -> (o, kappa, sign):
  // o | x << 13 | sign << 26
  std::vector<int> bk_ptr, bw_ptr;
  std::vector<unsigned> bk_ent, bw_ent;
  std::vector<int> out_of_state;  // sector state -> output index, -1 if none
};

template <typename E, typename F>
inline void group_csr(int ngroups, size_t n, F key_of, std::vector<int>& ptr, std::vector<E>& ent,
                      const std::vector<E>& val) {
  ptr.assign(ngroups + 1, 0);
  for (size_t e = 0; e < n; ++e) ptr[key_of(e) + 1]++;
  for (int g = 0; g < ngroups; ++g) ptr[g + 1] += ptr[g];
  ent.resize(n);
  std::vector<int> fill(ptr.begin(), ptr.end() - 1);
  for (size_t e = 0; e < n; ++e) ent[fill[key_of(e)]++] = val[e];
}

inline int build_adjoint(const Tables& T, AdjTables* A) {
  const int ns = T.nstate, no = T.nout;
  if (no >= (1 << 13) || ns >= (1 << 20) || T.nkey >= (1 << 15)) return -1;
  A->out_of_state.assign(ns, -1);
  for (int o = 0; o < no; ++o) A->out_of_state[T.out_state[o]] = o;
  // sector recursion
  {
    size_t ne = T.ent_sub.size();
    std::vector<int> owner(ne);
    for (int s = 0; s < ns; ++s)
      for (int e = T.ent_ptr[s]; e < T.ent_ptr[s + 1]; ++e) owner[e] = s;
    std::vector<unsigned long long> v1(ne), v2(ne);
    for (size_t e = 0; e < ne; ++e) {
      unsigned sl = (uint16_t)T.ent_slot[e];
      v1[e] = (unsigned long long)owner[e] | ((unsigned long long)sl << 32);
      v2[e] = (unsigned long long)owner[e] | ((unsigned long long)T.ent_sub[e] << 20) |
              ((unsigned long long)(sl & 1) << 40);
    }
    group_csr(ns, ne, [&](size_t e) { return T.ent_sub[e]; }, A->bs_ptr, A->bs_ent, v1);
    group_csr(T.nslot, ne, [&](size_t e) { return (int)((uint16_t)T.ent_slot[e] >> 1); }, A->bl_ptr, A->bl_ent, v2);
  }
  // output recursion: forward entries are indexed by level-order position
  {
    size_t ne = T.oent_sub.size();
    std::vector<int> owner(ne);
    for (size_t i = 0; i < T.olvl_order.size(); ++i)
      for (int e = T.oent_ptr[i]; e < T.oent_ptr[i + 1]; ++e) owner[e] = T.olvl_order[i];
    std::vector<int> pos_of_out(no);
    for (size_t i = 0; i < T.olvl_order.size(); ++i) pos_of_out[T.olvl_order[i]] = (int)i;
    std::vector<unsigned long long> v1(ne), v2(ne);
    for (size_t e = 0; e < ne; ++e) {
      unsigned sl = (uint16_t)T.oent_slot[e];
      v1[e] = (unsigned long long)owner[e] | ((unsigned long long)sl << 32);
      v2[e] = (unsigned long long)owner[e] | ((unsigned long long)T.oent_sub[e] << 20) |
              ((unsigned long long)(sl & 1) << 40);
    }
    // grouped by the level-order position of the sub output (kernels walk positions)
    group_csr(no, ne, [&](size_t e) { return pos_of_out[T.oent_sub[e]]; }, A->obs_ptr, A->obs_ent, v1);
    group_csr(T.nslot, ne, [&](size_t e) { return (int)((uint16_t)T.oent_slot[e] >> 1); }, A->obl_ptr, A->obl_ent,
              v2);
  }
  // Hamiltonian rows
  {
    size_t ne = T.h_s.size();
    std::vector<int> owner(ne);
    for (int o = 0; o < no; ++o)
      for (int e = T.h_ptr[o]; e < T.h_ptr[o + 1]; ++e) owner[e] = o;
    std::vector<unsigned> v1(ne);
    std::vector<unsigned long long> v2(ne);
    for (size_t e = 0; e < ne; ++e) {
      double cv = T.h_c[e];
      if (fabs(cv) != 1.0 && fabs(cv) != 0.5) return -2;
      unsigned neg = cv < 0, half = fabs(cv) == 0.5;
      v1[e] = (unsigned)owner[e] | ((unsigned)T.h_key[e] << 13) | (neg << 28) | (half << 29);
      v2[e] = (unsigned long long)owner[e] | ((unsigned long long)T.h_s[e] << 13) |
              ((unsigned long long)neg << 33) | ((unsigned long long)half << 34);
    }
    group_csr(ns, ne, [&](size_t e) { return T.h_s[e]; }, A->hs_ptr, A->hs_ent, v1);
    group_csr(T.nkey, ne, [&](size_t e) { return (int)T.h_key[e]; }, A->hk_ptr, A->hk_ent, v2);
  }
  // diagonal by key, E_0 by key
  {
    size_t ne = T.d_key.size();
    std::vector<int> owner(ne);
    for (int o = 0; o < no; ++o)
      for (int e = T.d_ptr[o]; e < T.d_ptr[o + 1]; ++e) owner[e] = o;
    std::vector<int> idx(ne);
    for (size_t e = 0; e < ne; ++e) idx[e] = (int)e;
    std::vector<int> grouped;
    group_csr(T.nkey, ne, [&](size_t e) { return (int)T.d_key[e]; }, A->dk_ptr, grouped, idx);
    A->dk_out.resize(ne);
    A->dk_c.resize(ne);
    for (size_t q = 0; q < ne; ++q) { A->dk_out[q] = owner[grouped[q]]; A->dk_c[q] = T.d_c[grouped[q]]; }
    A->e0_by_key.assign(T.nkey, 0.0);
    for (size_t e = 0; e < T.e0_key.size(); ++e) A->e0_by_key[T.e0_key[e]] += T.e0_c[e];
  }
  // back-substitution
  {
    // the row of output 0 is left out: the reference enters the Lagrangian as
    // phi'(ref) itself (the energy), never through a back-substituted R_0
    std::vector<unsigned> v1, v2;
    std::vector<int> kk_of, w_of;
    for (int o = 1; o < no; ++o)
      for (int e = T.b_ptr[o]; e < T.b_ptr[o + 1]; ++e) {
        unsigned sg = T.b_w[e] & 1, w = T.b_w[e] >> 1, kk = T.b_k[e];
        v1.push_back((unsigned)o | (w << 13) | (sg << 26));
        v2.push_back((unsigned)o | (kk << 13) | (sg << 26));
        kk_of.push_back((int)kk);
        w_of.push_back((int)w);
      }
    group_csr(no, v1.size(), [&](size_t e) { return kk_of[e]; }, A->bk_ptr, A->bk_ent, v1);
    group_csr(no, v2.size(), [&](size_t e) { return w_of[e]; }, A->bw_ptr, A->bw_ent, v2);
  }
  return 0;
}

inline const AdjTables* host_adjoint(int k, int K, int KH, int* rc) {
  static std::mutex mu;
  static std::unique_ptr<AdjTables> cache[kMaxSites + 1][4][5];
  const Tables* T = host_tables(k, K, KH, rc);
  if (!T) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  auto& slot = cache[k][K][KH];
  if (!slot) {
    std::unique_ptr<AdjTables> A(new AdjTables());
    *rc = build_adjoint(*T, A.get());
    if (*rc) return nullptr;
    slot = std::move(A);
  }
  return slot.get();
}

}  // namespace ph
