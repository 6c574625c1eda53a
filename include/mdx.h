/* mdx.h — C ABI of the GB300 McMurchie-Davidson electron-repulsion-integral engine.
 *
 * Method: Asadchev & Valeev, "3-center and 4-center 2-particle Gaussian AO
 * integrals on modern accelerated processors", arXiv:2405.01834.
 * Integrals are over contracted Cartesian Gaussian shells (Eq. 3) with
 * l <= MDX_LMAX, evaluated in FP64 by the McMurchie-Davidson scheme of Sec. 2
 * (Boys function, Eq. boys; auxiliary Hermite integrals, Eqs. 0m and r;
 * Hermite 2-index integrals, Eq. pq; ket then bra Hermite->Cartesian
 * transforms, Eqs. ket-from-hermite and bra-from-hermite).
 *
 * Conventions shared by every entry point
 *  - All array pointers are DEVICE pointers on the context's device, owned by
 *    the caller, and read-only unless stated. The library never frees caller
 *    memory. It allocates only inside the context (a workspace that grows on
 *    demand and is released by mdx_destroy).
 *  - Cartesian components of a shell of angular momentum l are ordered with
 *    a_x running from l down to 0, then a_y from l-a_x down to 0
 *    (xx, xy, xz, yy, yz, zz for l = 2).
 *  - Coefficients multiply the UNNORMALISED primitives
 *    x_A^ax y_A^ay z_A^az exp(-zeta r_A^2); any normalisation is folded in by
 *    the caller. Coordinates are in bohr.
 *  - Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL means
 *    the legacy default stream). Calls that must know the class mix of their
 *    input copy the (small) index arrays to the host and synchronise `stream`
 *    once before launching; each such call says so.
 *  - Every call validates its arguments on the host and returns a status; no
 *    C++ exception crosses the ABI. Errors detected inside a kernel (bad
 *    shell index, bounded wait expired) are recorded in a device error word of
 *    the context and returned by the next mdx_sync() or by the next call.
 *    mdx_last_error() gives a one-line description of the last failure.
 *  - A context is not thread-safe: calls on one context must not run
 *    concurrently from several host threads (use one context per thread).
 *    mdx_eri4_noalloc, which takes no context, serialises its host work on
 *    an internal lock.
 */
#ifndef MDX_H
#define MDX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MDX_LMAX 6          /* highest shell angular momentum */
#define MDX_KMAX 32         /* highest contraction degree of one shell */

typedef enum {
  MDX_OK = 0,
  MDX_EINVAL = 1,           /* bad argument (NULL pointer, negative size, shell index out of range) */
  MDX_ENOMEM = 2,           /* workspace allocation failed */
  MDX_ECUDA = 3,            /* a CUDA runtime call failed */
  MDX_EUNSUPPORTED = 4,     /* l > MDX_LMAX or contraction degree > MDX_KMAX */
  MDX_ECAPACITY = 5,        /* output buffer too small */
  MDX_ETIMEOUT = 6,         /* a bounded device-side wait expired */
  MDX_EDEVICE = 7,          /* a kernel flagged invalid input */
  MDX_ESCRATCH = 8          /* the request needs more than mdx_eri4_noalloc's fixed 32 MiB scratch */
} mdx_status;

typedef struct mdx_ctx mdx_ctx;

/* A basis of contracted Cartesian shells (Eq. 3). One entry per shell in l,
 * nprim, prim_off, ao_off, atom and center; one entry per primitive in exps
 * and coefs (shell s owns exps[prim_off[s] .. prim_off[s]+nprim[s]-1]).
 * ao_off[s] is the first AO (row of D and K) of shell s. atom may be NULL
 * except for mdx_exchange_grad. All pointers are device pointers. */
typedef struct {
  int32_t n_shells;
  int32_t n_prims;
  const int32_t* l;
  const int32_t* nprim;
  const int32_t* prim_off;
  const int32_t* ao_off;
  const int32_t* atom;
  const double* center;     /* [n_shells][3] */
  const double* exps;       /* [n_prims] */
  const double* coefs;      /* [n_prims] */
} mdx_basis;

/* Create a context on CUDA device `device` (made current for the call). The
 * context builds the Boys-function interpolation table and owns all
 * workspace. Returns MDX_OK and *ctx, or an error and *ctx = NULL. */
mdx_status mdx_create(mdx_ctx** ctx, int device);

/* Release the context and its workspace. NULL is allowed. The caller must
 * make sure no work the context enqueued is still running. */
void mdx_destroy(mdx_ctx* ctx);

/* Description of the last error of this context ("" if none). The string
 * lives until the next call on the context. */
const char* mdx_last_error(const mdx_ctx* ctx);

/* Synchronise `stream` and report (and clear) any error a kernel of this
 * context recorded in the device error word. */
mdx_status mdx_sync(mdx_ctx* ctx, void* stream);

/* 4-center integrals [ab|cd] (Eq. def-abcd) for n shell quartets.
 * quartets: [n][4] int32 shell indices (a, b, c, d) into `basis`.
 * bound: [n] doubles (device) or NULL. bound[q] is an upper bound on
 *   |(ab|cd)| over the shellset of quartet q, e.g. the Schwarz product
 *   Q_ab Q_cd of mdx_schwarz (the paper screens quartets before batching,
 *   Sec. 3, without fixing the bound). A quartet with bound[q] < tau is not
 *   evaluated: its shellset is written as zeros, its output slot and offset
 *   are unchanged. bound = NULL evaluates every quartet and ignores tau.
 * tau: screening threshold (>= 0 when bound is given, else MDX_EINVAL).
 * out: receives, for quartet q, the contracted shellset in row-major
 *   [a][b][c][d] order (d fastest) at out + out_offsets[q]; out has room for
 *   out_capacity doubles.
 * out_offsets: [n+1] int64, written by the call (exclusive prefix sum of the
 *   shellset sizes in quartet order); out_offsets[n] is the total.
 * Returns MDX_ECAPACITY (writing nothing) if the total exceeds out_capacity.
 * Copies the quartet list and the shell l/nprim arrays to the host and
 * synchronises `stream` to group quartets by class, then enqueues the kernels
 * and returns without waiting for them (results are ready when `stream`
 * reaches this point; errors their kernels record are returned by the next
 * call or mdx_sync). Its per-call device arrays are context workspace, never
 * cudaMalloc/cudaFree, so work on other streams is not stalled; calls of one
 * context that overlap must be issued on one stream. n = 0 is allowed and
 * writes out_offsets[0] = 0. */
mdx_status mdx_eri4(mdx_ctx* ctx, const mdx_basis* basis, const int32_t* quartets, const double* bound, int64_t n,
                    double tau, double* out, int64_t out_capacity, int64_t* out_offsets, void* stream);

/* mdx_eri4 over real solid harmonics (the paper's basis, Eqs. solid2herm-1/2):
 * a shell of angular momentum l contributes 2l+1 functions S_lm, m = -l..l,
 * S_lm = N_lm sum C x^.. y^.. z^.. with the standard real-solid-harmonic
 * coefficients, each with the angular norm of z^l (so x^l-normalised
 * contraction coefficients give normalised spherical functions; l = 1 is
 * (y, z, x)). Output per quartet [a][b][c][d] in solid-harmonic components at
 * out + out_offsets[q]; offsets and out_capacity count those doubles.
 * Classes evaluated by the team kernel contract the solid-harmonic
 * coefficients into the transforms, as the paper's H matrices do: the
 * Cartesian ket columns [p|cd] are staged in device memory (allocated by the
 * call), turned into [p|c'd'] one index at a time, and the bra steps and
 * everything after them run on 2l+1 components per shell. Small classes with
 * a register kernel are evaluated over Cartesians and transformed index by
 * index. Synchronises `stream`; results are complete on return. */
mdx_status mdx_eri4_sph(mdx_ctx* ctx, const mdx_basis* basis, const int32_t* quartets, int64_t n, double* out,
                        int64_t out_capacity, int64_t* out_offsets, void* stream);

/* 3-center integrals [a|cd] (Eq. def-acd): shell a from `aux`, shells c, d
 * from `orb`. triplets: [n][3] int32 (a, c, d). Output per triplet in
 * row-major [a][c][d] order at out + out_offsets[q]. The bra is a single
 * Gaussian (zeta_p = zeta_a, P = A) with the 1-center E coefficients of
 * Eq. E1rr. bound / tau: per-triplet bounds on |(a|cd)| (e.g. Q_a Q_cd) and
 * the threshold below which a triplet is written as zeros without being
 * evaluated, as in mdx_eri4 (bound = NULL: none). Same capacity, offset and
 * synchronisation rules as mdx_eri4. */
mdx_status mdx_eri3(mdx_ctx* ctx, const mdx_basis* aux, const mdx_basis* orb, const int32_t* triplets,
                    const double* bound, int64_t n, double tau, double* out, int64_t out_capacity,
                    int64_t* out_offsets, void* stream);

/* mdx_eri3 over real solid harmonics: [a|cd] (Eq. def-acd) with a, c and d
 * in solid-harmonic components (the bra's second function is the constant
 * s function, one component), [a][c][d] per triplet at out + out_offsets[q];
 * offsets and out_capacity count those doubles. Classes evaluated by the team
 * kernel use that a solid harmonic times a Gaussian expands in the top
 * Hermite shell |p| = l_a alone (the lower terms of Eq. E1rr cancel): only
 * those rows of [p|cd] are formed, the c and d indices are transformed as in
 * mdx_eri4_sph, and each component is (2 zeta_a)^-l_a sum_a C_ma [a|cd].
 * Small classes with a register kernel are evaluated over Cartesians and
 * transformed index by index. Synchronises `stream`; results are complete on
 * return. */
mdx_status mdx_eri3_sph(mdx_ctx* ctx, const mdx_basis* aux, const mdx_basis* orb, const int32_t* triplets, int64_t n,
                        double* out, int64_t out_capacity, int64_t* out_offsets, void* stream);

/* ---- prepared batches --------------------------------------------------
 * A batch separates the host-side preparation of a call (index download,
 * shell-pair de-duplication, grouping of quartets by class, planning,
 * uploads) from the launch of the hot path, so that one quartet list can be
 * evaluated repeatedly and its launches enqueued without host
 * synchronisation or allocation (e.g. inside a captured CUDA graph).
 * The basis descriptors' device arrays must stay valid until the batch is
 * destroyed; the batch keeps its own copies of the index data. */
typedef struct mdx_batch mdx_batch;

/* Prepare the quartets of mdx_eri4 (same arguments, without screening
 * bounds: a batch evaluates every quartet it is given). Synchronises
 * `stream`. n must be >= 1. */
mdx_status mdx_batch_eri4(mdx_ctx* ctx, const mdx_basis* basis, const int32_t* quartets, int64_t n,
                          mdx_batch** batch, void* stream);

/* Prepare the quartets of mdx_eri4_sph (same arguments): a batch whose
 * offsets, total and run output are in solid-harmonic components. Its device
 * arrays, including the staging of the solid-harmonic team kernel, belong to
 * the batch. Synchronises `stream`. n must be >= 1. mdx_batch_run_materialized
 * returns MDX_EUNSUPPORTED for such a batch; mdx_batch_autotune tunes its
 * solid-harmonic team-kernel classes (and may grow the staging area). */
mdx_status mdx_batch_eri4_sph(mdx_ctx* ctx, const mdx_basis* basis, const int32_t* quartets, int64_t n,
                              mdx_batch** batch, void* stream);

/* Prepare the triplets of mdx_eri3_sph (same arguments): a solid-harmonic
 * batch like those of mdx_batch_eri4_sph. Synchronises `stream`. */
mdx_status mdx_batch_eri3_sph(mdx_ctx* ctx, const mdx_basis* aux, const mdx_basis* orb, const int32_t* triplets,
                              int64_t n, mdx_batch** batch, void* stream);

/* Prepare the triplets of mdx_eri3 (same arguments). Synchronises `stream`. */
mdx_status mdx_batch_eri3(mdx_ctx* ctx, const mdx_basis* aux, const mdx_basis* orb, const int32_t* triplets,
                          int64_t n, mdx_batch** batch, void* stream);

/* Sizes of a prepared batch (host values; any pointer may be NULL): number of
 * quartets, output doubles, model FLOPs of the paper's Table 1 work model
 * adapted to contracted Cartesian shellsets, and FP64 multiply-adds the
 * engine issues. */
mdx_status mdx_batch_info(const mdx_batch* batch, int64_t* n, int64_t* total, double* model_flops,
                          double* exec_fma);

/* Copy the batch's [n+1] output offsets (see mdx_eri4) to out_offsets (device). */
mdx_status mdx_batch_offsets(mdx_ctx* ctx, const mdx_batch* batch, int64_t* out_offsets, void* stream);

/* Enqueue the whole evaluation of a batch on `stream`: primitive-pair records
 * (Eqs. E2rr1/E2rr2 or E1rr), then one quartet kernel per class (Eqs. boys,
 * 0m, r, pq, ket-from-hermite, bra-from-hermite). Writes the integrals at the
 * batch's offsets in `out` (out_capacity doubles). No host synchronisation
 * and no allocation; n_launches (may be NULL) receives the number of kernels
 * enqueued. Kernel-side errors surface at the next mdx_sync. */
mdx_status mdx_batch_run(mdx_ctx* ctx, mdx_batch* batch, double* out, int64_t out_capacity, int32_t* n_launches,
                         void* stream);

/* Autotuner (the analogue of the paper's per-class variant selection, Sec. 4):
 * for every class of the batch, time candidate team shapes (threads per
 * team, shared-memory budget per team, one or several ket-column groups) on
 * the first max_trial quartets of that class, keep the fastest for the
 * context (later batches of the class use it) and switch this batch to it.
 * Writes trial results into `out` (batch->total doubles needed) and
 * synchronises `stream`. Results are identical up to FP64 summation order.
 * Cartesian batches also time the register kernel where the class has one.
 * For a solid-harmonic batch: the classes that run the solid-harmonic team
 * kernel, over team sizes, shared-memory budgets and the cached R tables of
 * contracted classes, and the classes on the register-kernel route (Cartesian
 * shellsets, then the element-wise transform) against those team shapes
 * (MDX_ENOMEM if the chosen shape's staging area cannot be allocated).
 * Afterwards mdx_batch_info's exec_fma counts the shapes the batch runs. */
mdx_status mdx_batch_autotune(mdx_ctx* ctx, mdx_batch* batch, double* out, int64_t out_capacity,
                              int64_t max_trial, void* stream);

/* The same batch through the materialized-Hermite variant of the paper
 * (V2, Sec. 3): per quartet the full matrix [p|q] = (-1)^{|q|} [p+q] is written
 * to device memory and both transforms run as batched dense DGEMMs
 * ([p|cd] = [p|q] E^cd, [ab|cd] = E^ab [p|cd]; cuBLAS, i.e. the FP64 tensor
 * units). An A/B experiment against mdx_batch_run: same results, same output
 * layout, uncontracted 4-center classes only (MDX_EUNSUPPORTED otherwise),
 * synchronises the stream per class (not capturable). */
mdx_status mdx_batch_run_materialized(mdx_ctx* ctx, mdx_batch* batch, double* out, int64_t out_capacity,
                                      int32_t* n_launches, void* stream);

/* Free a batch (NULL allowed). No work of the batch may still be running. */
void mdx_batch_destroy(mdx_batch* batch);

/* Schwarz factors Q_ij = sqrt(max_ab |(ab|ab)|) over the Cartesian
 * components a of shell i and b of shell j, for n shell pairs. The paper
 * screens shell pairs before batching (Sec. 3, memory order of the batches)
 * without defining the bound; this is the standard Cauchy-Schwarz factor,
 * |(ab|cd)| <= Q_ab Q_cd, used by mdx_exchange's screening.
 * pairs: [n][2] int32 shell indices. Q_out: [n] doubles (device), written.
 * Works through the pairs in chunks whose diagonal shellsets hold at most
 * 2^27 doubles (1 GiB of workspace). Synchronises `stream`. */
mdx_status mdx_schwarz(mdx_ctx* ctx, const mdx_basis* basis, const int32_t* pairs, int64_t n,
                       double* Q_out, void* stream);

/* Hartree-Fock exchange K_ik = sum_jl D_jl (ij|kl) (Sec. 6 of the paper,
 * K_bc = sum_ad [ab|cd] D_ad with the indices renamed), no 1/2 or spin factor.
 * pairs: [n_pairs][2] int32 shell pairs, each unordered pair at most once
 *   (order inside a pair is free); Q: [n_pairs] Schwarz factors of the pairs
 *   (e.g. from mdx_schwarz), same order.
 * Unique quartets (ij|kl) of the pair list are screened on the GPU with
 *   Q_ij Q_kl max(|D_ik|, |D_il|, |D_jk|, |D_jl|) >= tau  (FP64; max over
 *   shell blocks; tau = 0 keeps every quartet). Pairs are sorted by Q within
 *   their class, so each bra pair stops testing a ket class at the first
 *   pair whose Q cannot pass; the cost follows the kept quartets, not the
 *   square of the pair count. The block maxima form one N_shells x N_shells
 *   table of doubles in context workspace. Each kept quartet is evaluated once
 *   and digested into four K blocks inside the integral kernel (the integrals
 *   never reach device memory), with FP64 atomics; finally K <- K + K^T.
 * D: [nao][nao] row-major, symmetric (device). K: [nao][nao] (device),
 *   overwritten. nao = max over shells of ao_off + ncart(l); basis->ao_off is
 *   required.
 * energy: one double (device) receiving the exchange energy
 *   E_x = alpha sum_ik D_ik K_ik = alpha sum_ijkl D_ik D_jl (ij|kl) of the
 *   screened K (alpha = -1 for a closed-shell D = C C^T), or NULL. Synchronises `stream` (screening counts) and on return K is
 *   complete. Pairs absent from the list contribute nothing. The per-class
 *   integral launches are spread over `stream` and three internal streams of
 *   the context, each ordered after the work already queued on `stream`, and
 *   `stream` waits for all of them before K <- K + K^T. */
mdx_status mdx_exchange(mdx_ctx* ctx, const mdx_basis* basis, const int32_t* pairs, const double* Q, int64_t n_pairs,
                        double tau, const double* D, double* K, double alpha, double* energy, void* stream);

/* The screening step of mdx_exchange on its own: the unique quartets
 * (ij|kl) of the pair list kept by Q_ij Q_kl max(|D_ik|,|D_il|,|D_jk|,|D_jl|)
 * >= tau (FP64, that product order; maxima over shell blocks of D).
 * *n_kept (host) receives their number; model_flops (host, may be NULL) the
 * paper's Table-1 work model summed over them (as mdx_batch_info counts it).
 * kept: [kept_capacity][2] int32 (device) or NULL for counting only;
 * receives each kept quartet as two indices into `pairs` (bra pair, ket
 * pair), grouped by class pair, in no particular order within a group.
 * MDX_ECAPACITY (with *n_kept set) when the list exceeds kept_capacity.
 * Pairs, Q, D and tau as in mdx_exchange. Synchronises `stream`. */
mdx_status mdx_exchange_screen(mdx_ctx* ctx, const mdx_basis* basis, const int32_t* pairs, const double* Q,
                               int64_t n_pairs, double tau, const double* D, int32_t* kept, int64_t kept_capacity,
                               int64_t* n_kept, double* model_flops, void* stream);

/* Nuclear gradient of the exchange energy E_x = alpha S, S = sum_ijkl D_ik D_jl
 * (ij|kl), with D held fixed (alpha = -1 for a closed-shell D = C C^T; the
 * paper lists geometric derivatives as future work, Sec. 7).
 * Same pairs, Q, tau and screening as mdx_exchange. For every kept unique
 * quartet the centres of three of its shells are differentiated through
 * the derivative of a primitive Cartesian Gaussian (Eq. 1),
 *   d/dA_x x_A^a e^(-zeta x_A^2) = 2 zeta x_A^(a+1) e - a x_A^(a-1) e,
 * i.e. classes with that shell's l raised (coefficients 2 zeta c) and lowered
 * by one, evaluated by the same Hermite machinery (Hermite index reaching
 * L+1) with [tuv] recomputed per launch, never stored, and contracted inside
 * the kernel with G = D_ik (x) D_jl + D_il (x) D_jk; the fourth centre follows
 * from translational invariance. Per class the fourth is the shell whose
 * raised and lowered classes cost most (an s shell has no lowered class).
 * basis->atom is required (atom of each shell, 0 <= atom < n_atoms).
 * Shells must have l <= MDX_LMAX - 1 (the raised classes reach l + 1);
 * MDX_EUNSUPPORTED otherwise (after the screening, before any integral
 * launch; grad is then left untouched).
 * grad: [n_atoms][3] doubles (device), overwritten with dE_x/dR (hartree/bohr
 * for normalised inputs). energy: one double (device) receiving E_x, or NULL.
 * The launches are spread over `stream` and the context's internal streams as
 * in mdx_exchange. Synchronises `stream`; results are complete on return. */
mdx_status mdx_exchange_grad(mdx_ctx* ctx, const mdx_basis* basis, const int32_t* pairs, const double* Q,
                             int64_t n_pairs, double tau, const double* D, double alpha, int32_t n_atoms,
                             double* grad, double* energy, void* stream);

/* ---- batched exchange of many molecules ---------------------------------
 * Exchange matrices K_m = sum_jl D_m,jl (ij|kl) of n_mol independent molecules
 * (uneven sizes, mixed classes and contraction degrees) prepared once and run
 * as one launch per integral class across all molecules, as one persistent
 * launch whose CTAs pull work items (a class's quartets for one block of
 * teams of the class's own team size, heaviest first) from a queue with a
 * single atomicAdd each, or as the register-kernel classes launched one by
 * one followed by one persistent launch over the remaining classes.
 * bases: host array of n_mol basis descriptors (device arrays, ao_off
 * required); D, K: host arrays of n_mol device pointers ([nao_m][nao_m]
 * row-major; D read, K overwritten by run). Every shell pair of every
 * molecule is used; its Schwarz factor is computed here, and unique quartets
 * are screened with Q_ij Q_kl max|D block| >= tau using each D as given at
 * creation. Synchronises `stream`. The D and K buffers must stay valid until
 * the batch is destroyed. */
typedef struct mdx_xbatch mdx_xbatch;
mdx_status mdx_xbatch_create(mdx_ctx* ctx, int32_t n_mol, const mdx_basis* bases, const double* const* D,
                             double* const* K, double tau, mdx_xbatch** xbatch, void* stream);

/* Kept quartets, persistent work items, per-class launches and the Table-1
 * model FLOPs of the kept shellsets of a batch (any pointer may be NULL). */
mdx_status mdx_xbatch_info(const mdx_xbatch* xbatch, int64_t* n_quartets, int64_t* n_items,
                           int32_t* n_class_launches, double* model_flops);

/* Enqueue K_m <- 0, the integral kernels with fused digestion and
 * K_m <- K_m + K_m^T. persistent = 0: one launch per class; 1: one persistent
 * launch over all classes (team kernel only); 2: one launch per class that
 * has a register kernel, then one persistent launch over the other classes.
 * Other values give MDX_EINVAL.
 * No host synchronisation and no allocation: the enqueued work can be
 * captured in a CUDA graph and replayed. n_launches (may be NULL) receives
 * the kernels enqueued. */
mdx_status mdx_xbatch_run(mdx_ctx* ctx, mdx_xbatch* xbatch, int32_t persistent, int32_t* n_launches, void* stream);

/* Autotuner of the per-class launches of a batched exchange (the analogue of
 * mdx_batch_autotune with the digestion epilogue): for every class launch,
 * time the register kernel (where the class has one) and team shapes (team
 * size; for classes of several column groups also the shared-memory budget
 * and the cached R tables) on its first max_trial quartets, keep the fastest
 * for the context and switch the batch's per-class launches to it. The
 * persistent work queue keeps the shapes it was built with. The trial
 * launches add into the K_m; the next mdx_xbatch_run zeroes them first.
 * Synchronises `stream`. */
mdx_status mdx_xbatch_autotune(mdx_ctx* ctx, mdx_xbatch* xbatch, int64_t max_trial, void* stream);

/* Per-class launch i of a batch (0 <= i < n_class_launches): its class
 * lk = {la, lb, lc, ld, K_ab, K_cd} (K = primitive pairs of the bra / ket
 * shell pairs), its kept quartets and their Table-1 model FLOPs (any output
 * pointer may be NULL). MDX_EINVAL for an index out of range. */
mdx_status mdx_xbatch_launch_info(const mdx_xbatch* xbatch, int32_t i, int32_t* lk, int64_t* n_quartets,
                                  double* model_flops);

/* Enqueue only the integral kernel (with fused digestion into the K_m) of
 * per-class launch i, without zeroing or symmetrising K_m: for timing one
 * class of a batch. Running every i between the zeroing and symmetrisation of
 * mdx_xbatch_run gives the same K_m. */
mdx_status mdx_xbatch_run_class(mdx_ctx* ctx, mdx_xbatch* xbatch, int32_t i, void* stream);

/* Free a batched exchange (NULL allowed). No work of it may still be running. */
void mdx_xbatch_destroy(mdx_xbatch* xbatch);

/* Number of unique quartets the last mdx_exchange of this context kept after
 * screening (-1 for a NULL context). */
int64_t mdx_last_quartet_count(const mdx_ctx* ctx);

/* mdx_eri4 without any device allocation, for callers that cannot let a
 * library call cudaMalloc: applications that own all device memory through
 * their own pool or budget and forbid allocations behind their back, and
 * steady-state loops that cannot afford cudaMalloc's implicit device
 * synchronisation. (The paper has no counterpart; this is a property of the
 * engine, not of the method.)
 * Same arguments and results as mdx_eri4 without screening bounds (every
 * quartet is evaluated) and minus the context: it runs on the
 * current CUDA device. All device scratch (Boys and Hermite decode tables,
 * primitive-pair records, quartet lists, class step programs) lives in one
 * file-scope 32 MiB __device__ array that every GPU loading the library holds
 * until the process exits. The first call on a device sets that device up
 * (looks up the array's address, fills the tables, synchronously); make that
 * first call before any stream capture. A request whose records, lists and
 * programs do not fit returns MDX_ESCRATCH and writes nothing. Every call
 * shares the one array and rewrites what it uses (the device error word is
 * cleared per call): calls that overlap on the GPU race and must not be
 * issued concurrently on different streams. Synchronises `stream`. No error
 * text is kept (no context): the status code is the report. */
mdx_status mdx_eri4_noalloc(const mdx_basis* basis, const int32_t* quartets, int64_t n, double* out,
                            int64_t out_capacity, int64_t* out_offsets, void* stream);

/* FP64 throughput of the current CUDA device, measured: the denominator of
 * the engine's roofline (the integral kernels are bound by the FP64 pipe).
 * The paper has no counterpart: it is a measurement utility of the engine.
 * kind 0: scalar FP64 fused multiply-add (DFMA), 8 independent chains per
 * thread; 1, 2, 3: the FP64 tensor-core instruction (mma.sync .f64) in the
 * shapes m8n8k4, m16n8k4 and m16n8k16, 4 independent accumulators per warp.
 * Register-resident loops over 8 blocks of 256 threads per SM; one warm-up
 * launch, then `reps` launches of about 100 ms timed with CUDA events on
 * `stream`. *gflops receives 2 x multiply-adds / second / 1e9. Synchronises
 * `stream`; allocates nothing. MDX_EINVAL for a kind outside 0..3, reps < 1
 * or a NULL gflops; MDX_ECUDA if a CUDA call fails. */
mdx_status mdx_fp64_peak(int kind, int reps, double* gflops, void* stream);

/* Shape the engine chooses for one integral class (no GPU needed; ctx may be
 * NULL). The class is (la lb | lc ld) with Kb = K_a K_b and Kk = K_c K_d
 * primitive pairs; one_centre = 1 selects the 3-center bra [a| (lb must be 0).
 * The planner applies the Hermite->Cartesian transforms of Eqs.
 * ket-from-hermite and bra-from-hermite one Cartesian axis at a time
 * (E factorises by axis, Sec. 2) and checks that every shared-memory access
 * of the resulting step programs stays inside the team workspace; a class
 * that cannot be planned returns MDX_EUNSUPPORTED.
 * exec_fma: FP64 multiply-adds the kernel issues per contracted shellset
 * (transforms, R recursion and Boys interpolation). */
typedef struct {
  int32_t team_threads;
  int32_t teams_per_cta;
  int32_t smem_bytes_per_team;
  int32_t n_groups;
  double exec_fma;
  int32_t register_kernel;   /* 1: store / digestion launches of the class use the register kernel */
  int32_t pad;
} mdx_plan_stats;

/* register_kernel: small classes have a kernel with one thread per quartet
 * (the paper's smallest variant V0, Sec. 3): total angular momentum <= 4 with
 * the Hermite table R, the [p|cd] block and the shellset in at most 100
 * registers' worth of doubles, and further classes of total angular momentum
 * <= 6 with R in registers and [p|cd] plus the shellset in shared memory. It
 * is the default for them, and the autotuner times it against the team
 * shapes. In gradient launches it evaluates the shifted shellsets into
 * workspace, and a separate kernel contracts them with D (x) D. */
mdx_status mdx_plan_info(mdx_ctx* ctx, int la, int lb, int lc, int ld, int Kb, int Kk, int one_centre,
                         mdx_plan_stats* out);

/* Fix the shape of one class for later calls of this context (what the
 * autotuner does after timing): team_threads (a power of two <= 1024, 0 for
 * the planner's choice), smem_budget (shared-memory bytes per team, 0 for the
 * default 200 KB) and variant (0: register kernel where the class has one,
 * else teams; 1: teams; 2: register kernel, MDX_EUNSUPPORTED when the class
 * has none; the solid-harmonic plan of the class takes the team shape and
 * always runs teams). Plans already built for the class are replaced; batches
 * prepared before keep theirs. */
mdx_status mdx_set_class_shape(mdx_ctx* ctx, int la, int lb, int lc, int ld, int Kb, int Kk, int one_centre,
                               int team_threads, int smem_budget, int variant);

#ifdef __cplusplus
}
#endif

#endif /* MDX_H */
