/*
 * ppq.h -- C ABI of the GB300 PQ / PH amplitude solver (perfect quadruples and
 * perfect hextuples models).
 *
 * The method (Theory section of the paper): coupled-cluster theory truncated
 * to amplitudes whose holes and particles carry at most K = 2 pairing labels
 * (CCSDTQ truncated to two pairs, Eq. decompose and Tables I-II), each label
 * P being the quartet of alpha/beta occupied orbital occ_of_pair[P] and
 * alpha/beta virtual orbital vir_of_pair[P] (Fig. 1: the k-th highest occupied
 * orbital paired with the k-th lowest virtual).  Two-electron integrals are
 * kept for at most two labels (Table I: v has rank-1 and rank-2 subtensors
 * only in PQ); the Fock matrix is the full one.  The projected equations
 * R_mu = <mu| exp(-T) H_N exp(T) |Phi> = 0 are evaluated exactly and solved
 * by Jacobi steps with orbital-energy denominators and DIIS (Implementation
 * section); the energy follows Eq. Ec.
 *
 * Amplitude layout (length ppq_amp_count):
 *   t1[P][k]     k = 0..2   single-pair excitations, P = 0..N-1
 *   t2[P][Q][k]  k = 0..28  two-pair excitations, stored for both orders of
 *                           the pair, t2[Q][P][swap(k)] = sign(k) t2[P][Q][k],
 *                           zero when P == Q (the paper's vanishing-diagonal
 *                           convention).
 * offset of t2 = 3N; ppq_amp_layout describes the excitation of each channel.
 * The three-pair (PH, K = 3) layout appends
 *   t3[P][Q][R][k]  k = 0..302  three-pair excitations at offset 3N + 29N^2,
 *                           stored for all six orders of the triple; a copy
 *                           with the labels and the channel's monomials
 *                           permuted alike carries (-1) for every transposed
 *                           pair of odd monomials; zero when two of P, Q, R
 *                           coincide.
 *
 * Conventions of every entry point
 *   - return 0 on success; < 0 on invalid arguments (nothing written, message
 *     in ppq_last_error); > 0 numerical status (1 not converged within
 *     max_iter, 2 diverged, 3 non-finite input) with outputs written; -9 when
 *     a tensor-core kernel's bounded wait timed out (see ppq_wait_selftest);
 *   - n_pairs >= 2; occ_of_pair / vir_of_pair are HOST int32 arrays of length
 *     n_pairs that together list every one of the 2 n_pairs active orbitals
 *     exactly once;
 *   - h (n_orb^2) and eri (n_orb^4, chemists' notation (pq|rs), 8-fold
 *     symmetric, row-major) are FP64 and may be host or device pointers
 *     (detected); they are read, never written, and stay caller-owned.  A
 *     pinned (page-locked, device-mapped) host eri is read in place by the
 *     kernels over the host link; pageable host memory is copied first;
 *   - amplitude / residual buffers are FP64 and may be host or device
 *     pointers (detected);
 *   - work runs on `stream` (a cudaStream_t, 0 = legacy default stream); the
 *     call returns after the stream has finished the work;
 *   - the library keeps a per-device workspace between calls (released by
 *     ppq_release); calls on one device are serialised by a mutex;
 *   - results are bit-reproducible: every reduction adds its partial sums in
 *     a fixed order.
 *
 * Arithmetic of the residual
 *   - precision 0 ("FP64"): every term in FP64, except that for n_pairs <= 80
 *     the quartic four-link term (Table V's heaviest class) runs on the tensor
 *     cores by exact integer splitting of its FP64 operands (42-bit fixed
 *     point per row / per integral block, 21 TF32 slice products with exact
 *     FP32 sums); its error is below ~3e-12 of (largest operand of the row) x
 *     (largest integral of the block) x n_pairs per element;
 *   - precision 1 ("FP32"): FP32 throughout, the quartic term as three TF32
 *     products (hi*hi + hi*lo + lo*hi), i.e. FP32 accuracy.
 */
#ifndef PPQ_H
#define PPQ_H
#include <stdint.h>
#include <stddef.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int K;              /* amplitude truncation: 2 = PQ (set by pq_solve; 3 by   */
                      /*     ph_solve)                                         */
  int K_H;            /* integral truncation in labels: 0 = same as K; pq_solve*/
                      /*     takes 2, ph_solve 2 or 3                           */
  int precision;      /* 0 = FP64 throughout; 1 = mixed: FP32 residual until   */
                      /*     ||R|| <= switch_tol or stagnation, then FP64      */
  double switch_tol;  /* 0 = the solver's default: 1e-4 for the dense PQ      */
                      /*     solver, 1e-5 for the label-subset solver (PH,     */
                      /*     K_H = -1); > 0 as given; < 0 is rejected          */
  double r_tol;       /* converged when ||R||_2 <= r_tol ...  (1e-10)           */
  double e_tol;       /* ... and |dE| <= e_tol (1e-10): dE between successive   */
                      /*     FP64 iterates, or (defect-correction polish) the   */
                      /*     energy change of one more Jacobi step, evaluated   */
                      /*     from the closures alone                            */
  int max_iter;       /* 200                                                   */
  int diis_dim;       /* 8 (0 disables DIIS)                                    */
  int diis_start;     /* 3                                                     */
  double level_shift; /* added to |denominator| (0)                             */
  int guess;          /* 0 = zero amplitudes, 1 = start from t_in, 2 (pq_solve, */
                      /*     pq_solve_cd) = start from the solution of the     */
                      /*     single-pair truncation (K = 1: amplitudes inside  */
                      /*     one pairing label, the perfect-pairing-type       */
                      /*     model), solved first by the label-subset solver   */
  int profile;        /* 1 = time every kernel with CUDA events on `stream`     */
                      /*     (ppq_profile_entry; pq_solve also fills            */
                      /*     t_quartic_ms, ... )                                */
  int polish;         /* after the switch (precision = 1): 0 = plain FP64       */
                      /*     Jacobi/DIIS iterations; 1 = FP64 defect correction:*/
                      /*     each outer step evaluates R in FP64 (norm, energy, */
                      /*     convergence test) and solves J d = -R with FP32    */
                      /*     finite-difference Jacobian products (default 1)    */
  int max_rank;       /* excitation-rank mask (Conclusions: higher excitations  */
                      /*     disabled, e.g. PH with singles and doubles only,   */
                      /*     a local CCSD): 0 = every rank; r = 1..6 keeps the  */
                      /*     amplitudes of excitation rank <= r and drops the   */
                      /*     residual equations of the others (the label-subset */
                      /*     solver: ph_solve, ph_solve_cd, ph_gradient, and    */
                      /*     pq_solve with K_H = -1); default 0                 */
} ppq_opts;

typedef struct {
  int status;          /* as the return value                                  */
  int iters;           /* residual evaluations (FP32 + FP64)                    */
  int polish_iters;    /* FP64 evaluations after the switch (mixed)            */
  int switched_at;     /* iteration of the precision switch (-1 none)          */
  double res_norm;     /* ||R||_2 over unique amplitudes at the returned t     */
  double e_corr;       /* correlation energy (Eh)                              */
  double e_total;      /* e_corr + reference energy + e_const (Eh)             */
  double t_residual_ms;/* device time in residual evaluations                  */
  double t_total_ms;   /* wall time of the call                                */
  double residual_flops; /* algorithmic FLOPs of one residual evaluation       */
  double quartic_flops;  /* algorithmic FLOPs of one launch of the quartic      */
                         /* (two-summed-label) contraction kernel              */
  double t_quartic_ms;   /* device time of those launches (profile = 1)        */
  int n_quartic;         /* number of those launches                           */
  int n_launches;        /* kernels launched by the call                       */
  int evals_fp32;        /* residual evaluations in FP32                        */
  int evals_fp64;        /* residual evaluations in FP64                        */
  double t_quartic32_ms; /* part of t_quartic_ms spent in FP32 launches         */
  int n_quartic32;       /* number of FP32 launches among n_quartic             */
} ppq_info;

/* Fill *o with the defaults listed above (the solver of the Implementation
   section: Jacobi steps with orbital-energy denominators and DIIS; the
   thresholds are this library's, the paper gives none).  Returns 0. */
int ppq_default_opts(ppq_opts* o);

/* Number of amplitudes of the layout above for n_pairs pairs: 3N + 29N^2
   for K = 2 (the <= 2-label manifold of Eq. decompose and Tables I-II:
   3N + 29 C(N,2) unique amplitudes, each two-pair one stored for both
   orders); 3N + 29N^2 + 303N^3 for K = 3 (plus 303 C(N,3) unique three-pair
   amplitudes, stored for all six orders).
   Returns 0, or -1 if K is not 2 or 3, or n_pairs < 1. */
int ppq_amp_count(int K, int n_pairs, size_t* n_amp);

/* Describe the channels of the block decomposition of T into pairing labels
   (Eq. decompose; pairs as in Fig. 1), K + 1 ints per channel.  K = 2: the
   32 channels (3 single-pair, then 29 two-pair), desc[3*c+0] = number of
   pairs (1 or 2), desc[3*c+1], desc[3*c+2] = 4-bit monomial masks of the
   first and second pair: bit 0 annihilates the alpha occupied orbital,
   bit 1 the beta occupied, bit 2 creates the alpha virtual, bit 3 the beta
   virtual.  The excitation operator of t1[P][k] is E_P^{m}; that of
   t2[P][Q][k] is E_P^{a} E_Q^{b}, with E^m = (a+_{v,alpha})^{b2}
   (a+_{v,beta})^{b3} (a_{o,beta})^{b1} (a_{o,alpha})^{b0} on one pair.
   K = 3: the same 32 channels then the 303 three-pair ones (Table II's
   three-label blocks), desc[4*c+0] = number of pairs (1, 2 or 3) and three
   monomials; t3[P][Q][R][k] has the operator E_P^{a} E_Q^{b} E_R^{c}.
   desc must hold 96 ints for K = 2 and 1340 for K = 3.  Returns 0, or -1
   if K is not 2 or 3. */
int ppq_amp_layout(int K, int* desc);

/* One residual evaluation R(T) and correlation energy at amplitudes t (both
   in the layout above): the operation of the Theory section, Eq. decompose
   inserted into the projected CC equations.  precision 0 = FP64, 1 = FP32
   contractions (energy sums in FP64). */
int pq_residual(int n_pairs, const int* occ_of_pair, const int* vir_of_pair,
                const double* h, const double* eri, const double* t,
                double* r, double* e_corr, int precision, void* stream);

/* Solve the PQ amplitude equations (Theory section) by Jacobi steps with
   orbital-energy denominators and DIIS (Implementation section); the energy
   is Eq. Ec.  opts->K_H = 0 or 2 runs the two-label PQ kernels; -1 keeps every
   two-electron integral and runs the label-subset solver of ph_solve with
   K = 2 (n_pairs <= 127).  t_in (nullable unless guess == 1) and
   t_out use the layout above; e_corr / e_total / info are host pointers
   (nullable).  e_total = e_corr + E_ref + e_const with
   E_ref = sum_i (h_ii + f_ii) over the occupied orbitals. */
int pq_solve(int n_pairs, const int* occ_of_pair, const int* vir_of_pair,
             const double* h, const double* eri, double e_const,
             const ppq_opts* opts, const double* t_in, double* t_out,
             double* e_corr, double* e_total, ppq_info* info, void* stream);

/* One residual evaluation of the PH model (the three-pair truncation, K = 3:
   singles through hextuples over at most three pairing labels; Theory
   section, Table II) at amplitudes t in the K = 3 layout above, with the
   two-electron integrals truncated to at most K_H labels (K_H = 0 or 3: the
   rank-3 subtensors of v of Table I; 2: two labels).  Only the sorted-label
   entries of t (t2[P][Q] with P < Q, t3[P][Q][R] with P < Q < R) are read; r
   receives every stored order (copies by the layout's rule, zero where labels
   repeat).  Exact evaluation: the residual is assembled from local problems
   over every label subset of at most K + K_H labels, each solved in its
   site basis (psi = exp(T)|ref>, <kappa| H |psi>, back-substitution with
   exp(-T)), with inclusion-exclusion coefficients; a linked term of the
   projected equations never carries more than K + K_H labels.
   h, eri, t, r host or device pointers (detected); e_corr host (nullable).
   precision 0 = FP64, 1 = FP32 local problems (assembly and energy sums in
   FP64).  n_pairs <= 127.  Returns 0 or < 0 on invalid arguments. */
int ph_residual(int n_pairs, const int* occ_of_pair, const int* vir_of_pair,
                const double* h, const double* eri, const double* t, double* r,
                double* e_corr, int precision, int K_H, void* stream);

/* Solve the PH amplitude equations (Theory section, K = 3) by Jacobi steps
   with orbital-energy denominators and Pulay DIIS (Implementation section),
   with the arguments and conventions of pq_solve; t_in / t_out use the K = 3
   layout.  opts->K is ignored (the entry point sets K = 3); opts->K_H = 0 or
   3 keeps three-label integrals, 2 keeps two.  precision 1 runs FP32
   residuals until ||R|| <= switch_tol or stagnation, then FP64 to the final
   tolerances: with opts->polish = 1 (default) by defect correction (each
   outer step evaluates R in FP64 and solves J d = -R with forward-difference
   Jacobian products of FP32 residuals), with 0 by plain FP64 Jacobi/DIIS,
   which it also falls back to when an outer step gains less than 10x or
   ||R|| <= r_tol.  The DIIS least-squares
   problem is solved on the device; the host reads ||R|| and E_c once per
   iteration.  info->residual_flops counts 2 FLOPs per table entry and label
   subset of one residual evaluation.  n_pairs <= 127.
   The first call for a subset size builds that size's structure tables on
   the host (about 6 s and 0.7 GB for six labels) and keeps them on the device
   (about 1 GB for six labels) until the process exits. */
int ph_solve(int n_pairs, const int* occ_of_pair, const int* vir_of_pair,
             const double* h, const double* eri, double e_const,
             const ppq_opts* opts, const double* t_in, double* t_out,
             double* e_corr, double* e_total, ppq_info* info, void* stream);

/* One residual evaluation by the label-subset expansion (the evaluation of
   ph_residual) for amplitudes over at most K = 2 or 3 pairing labels (Theory
   section, Eq. decompose) and two-electron integrals over at most K_H labels:
   K_H = 0 (= K), 2, 3, or -1 = untruncated (K = 2 only: then a linked term
   carries up to K + 4 = 6 labels; the paper's integral truncation controlled
   separately from the amplitudes, Implementation section).  Layout, pointers
   and errors as ph_residual, with the layout of K (3N + 29N^2 for K = 2).
   pq_solve runs this evaluation for opts->K_H = -1. */
int ppq_subset_residual(int K, int K_H, int n_pairs, const int* occ_of_pair, const int* vir_of_pair,
                        const double* h, const double* eri, const double* t, double* r,
                        double* e_corr, int precision, void* stream);

/* Host-only export of the structure tables that ph_residual generates for
   local problems of k sites (amplitudes over at most K labels, integrals over
   at most K_H): the zero-charge sector, the recursions of exp(+-T)|ref>, the
   Hamiltonian rows and the back-substitution.  The paper has no counterpart:
   this is how the library lays out the exact evaluation, exported so that a
   CPU check can interpret the tables against the oracle.  ph_tables_counts
   fills counts[0..46] (counts must hold 48) with the element count of each
   table; ph_tables_copy copies table `which` (0..46) into dst (host memory of
   counts[which] elements: uint32 codes; int32 pointers, indices and
   descriptors; int16 slot / key fields; double coefficients; 26..46 are the
   transposed (adjoint) tables of the Lambda / gradient pass, with uint64 or
   uint32 packed entries).  No device call.  Returns 0, or < 0 for k outside 1..6 or K, K_H outside 1..3. */
int ph_tables_counts(int k, int K, int K_H, int64_t* counts);
int ph_tables_copy(int k, int K, int K_H, int which, void* dst);

/* pq_solve and ph_solve with the two-electron integrals given as three-index
   factors, (pq|rs) = sum_Q B[Q][p][q] B[Q][r][s] (Cholesky or RI vectors; the
   paper builds its integral blocks from such B matrices, Implementation
   section, with a Cholesky threshold in the Results section).  B is FP64,
   naux x n_orb x n_orb row-major, host or device (detected), read only; the
   dense n_orb^4 array is never formed: the Fock matrix and every gathered
   integral block are contracted from B on the device (B is transposed once
   into a [pq][Q] working copy of the same size).  Other arguments, statuses
   and outputs as pq_solve / ph_solve; pq_solve_cd accepts opts->K_H = -1. */
int pq_solve_cd(int n_pairs, const int* occ_of_pair, const int* vir_of_pair,
                const double* h, const double* B, int naux, double e_const,
                const ppq_opts* opts, const double* t_in, double* t_out,
                double* e_corr, double* e_total, ppq_info* info, void* stream);
int ph_solve_cd(int n_pairs, const int* occ_of_pair, const int* vir_of_pair,
                const double* h, const double* B, int naux, double e_const,
                const ppq_opts* opts, const double* t_in, double* t_out,
                double* e_corr, double* e_total, ppq_info* info, void* stream);

/* Solve n_sys independent PQ problems of (possibly different) sizes in one
   call: the batched form of the paper's calculations, e.g. a bond-length scan
   of H50-like chains (Results section).  Per system i: n_pairs[i],
   occ_of_pair[i] / vir_of_pair[i] (host), h[i], eri[i] (host or device),
   e_const[i] (nullable array), t_out[i] (nullable array of nullable
   pointers); e_corr / e_total / info are host arrays of n_sys (nullable).
   Every system starts from zero amplitudes with the same opts.  The systems
   run concurrently on a pool of worker threads (PPQ_BATCH_THREADS, default
   8), each with its own stream and cached workspace; every workspace replays
   its residual pipeline as a captured CUDA graph, and the quartic GEMM tile
   is autotuned once per pair count.  The batch starts after the work already
   queued on `stream` and the call returns when every system is done.
   Returns < 0 on invalid arguments, else the largest per-system status
   (0 when all converged); per-system statuses are in info[i].status. */
int pq_solve_batched(int n_sys, const int* n_pairs, const int* const* occ_of_pair,
                     const int* const* vir_of_pair, const double* const* h,
                     const double* const* eri, const double* e_const, const ppq_opts* opts,
                     double* const* t_out, double* e_corr, double* e_total, ppq_info* info,
                     void* stream);

/* Gradient of the Lagrangian L(t, lambda) = E_c(t) + sum_mu lambda_mu R_mu(t)
   with respect to the amplitudes at arbitrary (t, lambda) (both in the
   amplitude layout, two-pair copies consistent): grad = dE_c/dt + J^T lambda,
   evaluated by the reverse-mode (adjoint) kernels with the transposed
   contraction structure of the residual (Theory section: lambda lives on the
   same truncated manifold as t, Table I).  grad is written in the same layout
   (both copies of a two-pair entry hold the derivative with respect to the
   one independent amplitude).  FP64.  e_corr (host, nullable) receives E_c(t). */
int pq_lagrangian_gradient(int n_pairs, const int* occ_of_pair, const int* vir_of_pair,
                           const double* h, const double* eri, const double* t,
                           const double* lam, double* grad, double* e_corr, void* stream);

/* Solve the Lambda (left) equations grad_t L(t, lambda) = 0 at converged
   amplitudes t (the left-hand amplitudes live on the same truncated manifold
   as t, Theory section and Table I): Jacobi steps lambda += grad / D with
   DIIS, FP64, converged when ||grad||_2 <= opts->r_tol (max_iter steps).  lam_out uses the amplitude
   layout.  Returns 0, 1 (not converged) or 2 (diverged), or < 0 on errors. */
int pq_lambda(int n_pairs, const int* occ_of_pair, const int* vir_of_pair, const double* h,
              const double* eri, const double* t, const ppq_opts* opts, double* lam_out,
              ppq_info* info, void* stream);

/* Energy gradients of the PQ model (Theory section; the response of the
   energy to h and (pq|rs) through the Lambda equations on the Table I
   manifold): solve the amplitudes (opts as pq_solve, from zero), solve
   Lambda (FP64), then form dE_total/dh (n_orb^2), dE_total/d(pq|rs) (n_orb^4) and the
   orbital-rotation gradient dE/dkappa (n_orb^2, antisymmetric) for
   C -> C exp(kappa) with the pairing kept by index.  The integral gradients
   are symmetrised: dE = sum G delta for symmetric perturbations delta (all
   copies of an integral perturbed together).  E_total includes E_ref and
   e_const, so the gradients include their explicit dependence.  Every
   output is nullable and may be host or device memory.  Returns the larger
   of the amplitude and Lambda statuses, or < 0 on errors. */
int pq_gradient(int n_pairs, const int* occ_of_pair, const int* vir_of_pair, const double* h,
                const double* eri, double e_const, const ppq_opts* opts, double* t_out,
                double* lam_out, double* dE_dh, double* dE_deri, double* dE_dkappa,
                double* e_total, ppq_info* info, void* stream);

/* grad_t L(t, lambda) of the PH model (K = 3; K_H = 0 or 3: three-label
   integrals, 2: two-label), the Lagrangian L = E_c + sum over unique mu of
   lambda_mu R_mu (Theory section: lambda on the truncated manifold of t).
   t and lam use the K = 3 layout (ppq_amp_count(N, 3) doubles, host or
   device; only the sorted-label entries are read).  The reverse pass runs
   through every local problem of the label-subset expansion (transposed
   structure tables, FP64) and sums each adjoint over the subsets containing
   its labels in a fixed order: the result is reproducible.  grad is written
   in the same layout, copies filled by the copy rule.  e_corr (host,
   nullable) receives E_c(t).  Returns 0 or < 0 (-4 bad K_H, -2 null buffer,
   -1 bad pairing or n_pairs > 127). */
int ph_lagrangian_gradient(int n_pairs, const int* occ_of_pair, const int* vir_of_pair,
                           const double* h, const double* eri, const double* t,
                           const double* lam, int K_H, double* grad, double* e_corr, void* stream);

/* Energy gradients of the PH model: solve the amplitudes (opts as ph_solve,
   from zero amplitudes), then the Lambda equations grad_t L = 0 (FP64 Jacobi steps
   with device DIIS, from zero, to opts->r_tol), then the relaxed integral
   gradients from the adjoints of every gathered integral, transposed to
   dense dE_total/dh (n_orb^2) and dE_total/d(pq|rs) (n_orb^4) through the
   chain rule of the bare one-body part and of E_ref, and the
   orbital-rotation gradient dE/dkappa (n_orb^2) as pq_gradient.  eri must be
   dense.  Outputs nullable, host or device; t_out and lam_out in the K = 3
   layout.  Returns the larger of the amplitude and Lambda statuses, or < 0. */
int ph_gradient(int n_pairs, const int* occ_of_pair, const int* vir_of_pair, const double* h,
                const double* eri, double e_const, const ppq_opts* opts, double* t_out,
                double* lam_out, double* dE_dh, double* dE_deri, double* dE_dkappa,
                double* e_total, ppq_info* info, void* stream);

/* pq_residual without any device allocation.  The paper has no counterpart:
   this entry point exists for callers that cannot call cudaMalloc.  Examples
   are code running inside another framework's memory pool or under a fixed
   device-memory budget, or code on a path where cudaMalloc's implicit device
   synchronisation is not acceptable.  Every intermediate lives in one
   file-scope device array of 8 MiB, sized for at most 12 pairs (the
   intermediates grow as n_pairs^2 and take 4.4 MiB at 12 pairs).  Each GPU
   that loads the library holds that array until the process exits; larger
   sizes return -6 with a message.
   h, eri, t and r must be device pointers (else -7); occ_of_pair / vir_of_pair
   are host arrays; e_corr is a host pointer (nullable).  The quartic term uses
   the SIMT kernel with a fixed tile (no autotuning).  The call is synchronous:
   it returns after `stream` has finished its work, also on an error after
   work was queued.  The first call on a device looks up the array's device
   address (cudaGetSymbolAddress) while that device is current; make that
   first call before any stream capture.  Each call clears the part of the
   array it uses before use.  Calls from this library are serialised by its
   mutex and by that final synchronisation; kernels of two calls could only
   overlap on the GPU if a caller bypassed both (for example by queuing the
   array's users from another library copy), and such overlapping calls race
   on the array. */
int pq_residual_static(int n_pairs, const int* occ_of_pair, const int* vir_of_pair,
                       const double* h, const double* eri, const double* t,
                       double* r, double* e_corr, int precision, void* stream);

/* Natural occupation numbers (Results section: the occupations that measure
   static correlation, e.g. of the acenes): the eigenvalues, in descending
   order, of a symmetric one-particle density matrix gamma (n_orb x n_orb, FP64,
   host or device; the relaxed density dE_total/dh returned by pq_gradient is
   one), by cyclic Jacobi rotations in one thread block on the device.
   occ_out receives n_orb values; vecs_out (nullable) the natural orbitals as
   columns (n_orb x n_orb, row-major).  n_orb <= 160 (<= 120 with vecs_out).
   Synchronous on `stream`.  Returns 0 or < 0 on invalid arguments. */
int ppq_natural_occupations(int n_orb, const double* gamma, double* occ_out, double* vecs_out, void* stream);

/* Self-test of the bounded waits (library housekeeping; the paper has no
   counterpart).  The tensor-core kernels bound every mbarrier wait (about 1 s);
   on a timeout they stop issuing work, drain what they issued, flag the error
   and poison their output, and the solvers then return -9 with a message
   instead of a number.  This call runs the same bounded wait on a barrier
   that nothing arrives on, with a limit of `cycles` clock cycles (1 .. 4e9),
   and sets *timed_out = 1 when the wait ran out (the expected outcome); no
   copy, MMA or tensor memory is involved.  Returns 0, or < 0 on errors. */
int ppq_wait_selftest(long long cycles, int* timed_out, void* stream);

/* Free the cached workspace of the current device (library housekeeping;
   the paper has no counterpart).  Returns 0. */
int ppq_release(void);

/* Thread-local message of the last failing call on this thread ("" if none;
   library housekeeping, the paper has no counterpart). */
const char* ppq_last_error(void);

/* Per-kernel device time of the last call made with opts->profile = 1
   (library instrumentation; the paper has no counterpart).  CUDA events are
   recorded on the call's stream after every kernel, and each kernel class is
   charged the stream time since the previous event, so the classes add up to
   the stream time of the call.  ppq_profile_count returns the number of
   classes (waiting for the recorded events); ppq_profile_entry(i, ...) fills
   the class name (NUL-terminated, at most name_cap bytes), milliseconds,
   launches, algorithmic bytes and FLOPs of class i (every output nullable).
   Returns 0, or -2 for an index out of range. */
int ppq_profile_count(void);
int ppq_profile_entry(int i, char* name, int name_cap, double* ms, int* launches, double* bytes,
                      double* flops);

/* Work list of the tensor-core form of the quartic topology (Sec. II, the
   four-link term of the linked residual) for n_pairs <= 80; host only, no
   device call.  The paper has no counterpart: it is how this library tiles the
   term on the GPU.  A chunk is one link pair (c1, c2) with up to four
   Hamiltonian components g: 12 int16 fields
     c1, c2, n_g, n_cols (= n_g * 16 ceil(n_pairs / 16)), g[4], q[4]
   (q = index of the (c1, c2, g) combination, unused slots 0).  A CTA record
   is 3 ints: row tile (128 unordered pairs Y < Z, in order of Y then Z),
   first chunk, end chunk.  chunks (room for max_chunks records) and ctas
   (room for max_ctas records) may be NULL to query the counts; n_chunks and
   n_ctas receive them.  Returns 0, -2 (too little room) or -5 (n_pairs out of
   range). */
int ppq_tc_plan(int n_pairs, int16_t* chunks, int max_chunks, int* ctas, int max_ctas, int* n_chunks,
                int* n_ctas);

#ifdef __cplusplus
}
#endif
#endif
