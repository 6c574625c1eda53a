// Launch interface between the host API and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>

#include "mdx_internal.h"

namespace mdx {

struct BasisDev {
  const int32_t* l;
  const int32_t* nprim;
  const int32_t* prim_off;
  const double* center;
  const double* exps;
  const double* coefs;
};

// One primitive-pair record to build: shells (i, j) of basis `which`
// (j < 0: one-centre bra, partner is the unit function phi = 1), primitive
// indices (ia, ib), and the record's offset (doubles) in the record arrays.
struct PrimPairJob {
  int32_t i, j, ia, ib;
  int32_t which, pad;
  int64_t off;
};

// Device error codes recorded in the context's error word.
enum DevErr : int { kDevOk = 0, kDevBadInput = 1, kDevTimeout = 2 };

cudaError_t launch_pair_records(const BasisDev& b0, const BasisDev& b1, const PrimPairJob* jobs, int64_t njobs,
                                double* recs, double* recs_signed, int* err, cudaStream_t s);

struct QuartetLaunch {
  PlanDev plan;
  int64_t nq;
  const int2* qpairs;        // (bra pair, ket pair) per quartet
  const int64_t* qout;       // output offset (doubles) per quartet
  const int64_t* pair_rec;   // first record of each pair
  const double* recs;
  const double* recs_signed;
  const double* boys;
  const uint32_t* rprog;     // R-level programs (one word per Hermite entry, build_rlevel_programs)
  const int32_t* rprog_off;  // start of each total order N in rprog
  double* out;
  int* err;
  // exchange digestion (out unused when D != nullptr): K_ik += w sum_jl D_jl (ij|kl)
  // and the three other index placements of the unique quartet (see k_quartets)
  const double* D;
  double* K;
  int32_t nao;
  const int32_t* ao_off;     // per shell, of the basis of the pairs
  const int2* pair_shells;   // per pair (i, j)
  // record variants: quartet (p, q) reads the records of pairs p + bra_var_off and q + ket_var_off
  int64_t bra_var_off, ket_var_off;
  // exchange gradient (grad != nullptr): this launch evaluates the class with the shell at
  // position gpos (0: i, 1: j, 2: k, 3: l) replaced by its l+1 (gsign = +1, coefficients 2 zeta c) or
  // l-1 (gsign = -1) partner and contracts with G = D_ik D_jl + D_il D_jk; gpos = -1: the energy.
  // The atom of the shell at position ginv (never gpos) takes minus what gpos gains.
  double* grad;              // [n_atoms][3]
  double* energy;
  const int32_t* atom;       // per shell
  double alpha;
  int32_t gpos, gsign, ginv;
  int32_t lorig[4];          // unshifted l of positions i, j, k, l
  // several molecules in one launch (exchange): molecule of each pair and its D, K, nao
  const int32_t* pair_mol;
  const double* const* mol_D;
  double* const* mol_K;
  const int32_t* mol_nao;
  // solid-harmonic launches (plan.sph): global staging, xg_doubles per team of the launch grid
  double* sph_scratch;
};

static_assert(sizeof(QuartetLaunch) % sizeof(int) == 0, "descriptor copied word by word");

// Persistent launch over work items of many QuartetLaunch descriptors.
constexpr int kPersistBlock = 512;
constexpr int64_t kPersistSmem = 110 * 1024;   // shared memory per persistent block (two blocks per SM)
constexpr int kPersistRounds = 4;              // rounds of teams per work item
struct WorkItem {
  int32_t launch;   // index into PersistLaunch::launches
  int32_t count;    // quartets of this item (rounds of one quartet per team)
  int64_t begin;    // first quartet (index into that launch's qpairs)
};
struct PersistLaunch {
  const QuartetLaunch* launches;   // device array
  const WorkItem* items;           // device array, heaviest first
  int64_t nitems;
  unsigned long long* counter;     // next item; zero before the launch
};
cudaError_t launch_persistent(const PersistLaunch& pl, int64_t smem_bytes, int grid, cudaStream_t s);
const void* persistent_kernel_ptr();

cudaError_t launch_quartets(const QuartetLaunch& a, cudaStream_t s);
// Solid-harmonic shellsets (plan.sph, store at a.out + a.qout[q]): `grid` CTAs loop over the quartets;
// sph_grid gives the grid for nq quartets (resident CTAs at most), and a.sph_scratch must hold
// grid * teams_per_cta * xg_doubles doubles.
cudaError_t sph_grid(const PlanDev& P, int64_t nq, int* grid);
cudaError_t launch_quartets_sph(const QuartetLaunch& a, int grid, cudaStream_t s);
// Writes zeros over n output ranges given as (offset, doubles) pairs (screened-out shellsets).
cudaError_t launch_zero_ranges(const int64_t* ranges, int64_t n, double* out, cudaStream_t s);
// Gradient epilogue over shellsets already in memory (V + q N_b N_k for quartet q of launch a).
cudaError_t launch_grad_contract(const QuartetLaunch& a, const double* V, cudaStream_t s);

// Exchange support: per shell-pair block max |D| (FP64), per-shell row maxima
// of that table, screening of unique quartets into class buckets, K <- K + K^T.
cudaError_t launch_dmax(const double* D, int32_t nao, const int32_t* ao_off, const int32_t* l, int32_t n_shells,
                        double* dmax, int64_t ld, cudaStream_t s);
// rowmax[i] = max_k dmax[i * n + k] for the n shells of one table
cudaError_t launch_rowmax(const double* dmax, int32_t n, double* rowmax, cudaStream_t s);
// Unique quartets (p, q) of a pair list kept when Q_p Q_q max(|D_ik|,|D_il|,|D_jk|,|D_jl|) >= tau,
// evaluated in FP64 exactly in that order. Pairs are grouped into segments of one molecule and one
// pair class, each listed in `order` by decreasing Q; q runs over the segments of p's molecule whose
// class is <= p's class (in its own segment up to p's position), so every unordered pair of pairs is
// tested once. A binary search stops each segment where Q_p Q_q rowmax < tau (every later q of the
// descending segment fails too, since the product is monotone in Q_q and the block maximum is at most
// the row maximum).
struct ScreenArgs {
  int64_t npairs;
  const int2* pair_shells;     // per pair (i, j)
  const double* Q;             // Schwarz factor per pair
  const int32_t* pair_class;   // class index per pair
  const int64_t* pos;          // position of each pair in `order`
  const int32_t* order;        // pair indices, segment by segment, Q decreasing within a segment
  const int64_t* seg_begin;    // [nseg + 1] first position of each segment in `order`
  const int32_t* seg_class;    // class of each segment (increasing within a molecule)
  const int32_t* mol_seg;      // [nmol + 1] first segment of each molecule
  const int32_t* pair_mol;     // molecule of each pair (NULL: one molecule)
  const int32_t* shell_first;  // [nmol + 1] first shell of each molecule
  const int64_t* dmax_off;     // [nmol] start of each molecule's [n_m][n_m] table in dmax
  const double* dmax;
  const double* rowmax;        // per shell (global shell numbering)
  int32_t nclass;
  double tau;
  unsigned long long* counts;  // [nclass*(nclass+1)/2] bucket (cp, cq), cp >= cq, at cp*(cp+1)/2 + cq
  const int64_t* bucket_off;   // fill pass: start of each bucket
  int2* out;                   // fill pass: (p, q) per surviving quartet
};
cudaError_t launch_screen(const ScreenArgs& a, bool fill, cudaStream_t s);
// out[2k], out[2k+1] = orig[qp[k].x], orig[qp[k].y] (sorted pair indices back to caller indices)
cudaError_t launch_map_pairs(const int2* qp, int64_t n, const int64_t* orig, int32_t* out, cudaStream_t s);
cudaError_t launch_symmetrize(double* K, int32_t nao, cudaStream_t s);
// *energy += alpha sum_i D[i] K[i] over n doubles (the caller zeroes *energy)
cudaError_t launch_dot_energy(const double* D, const double* K, int64_t n, double alpha, double* energy,
                              cudaStream_t s);
// K <- 0 (zero = true) or K <- K + K^T (zero = false) for nmol molecules; K and nao are device arrays
cudaError_t launch_multi_k(double* const* K, const int32_t* nao, int32_t nmol, int64_t max_nao, bool zero,
                           cudaStream_t s);
cudaError_t kernel_attributes_init();

// Cartesian -> real solid harmonic transform of one class of 4-center shellsets.
struct SphLaunch {
  int32_t la, lb, lc, ld;
  int64_t nq;
  const double* cart;        // Cartesian shellsets
  const int64_t* coff;       // per shellset: offset in cart
  double* out;               // solid-harmonic shellsets [a'][b'][c'][d'], m = -l..l
  const int64_t* ooff;
};
cudaError_t launch_cart2sph(const SphLaunch& a, cudaStream_t s);

// Materialized-Hermite path (A/B experiment): E matrices of listed pairs
// (bra: [N_b x Nt(L)] rows ab; ket: [Nt(L) x N_k] rows q), [p|q] matrices of a
// chunk of quartets, and the pointer arrays of the two batched products.
cudaError_t launch_mat_emat(const double* recs, const int64_t* pair_rec, const int32_t* pairs, int64_t npairs,
                            int la, int lb, bool bra, double* E, cudaStream_t s);
cudaError_t launch_mat_hermite(const double* recs, const int64_t* pair_rec, const int2* qp, int64_t nq, int Lb,
                               int Lk, const double* boys, double* PQ, cudaStream_t s);
cudaError_t launch_mat_ptrs(int64_t nq, const int32_t* ib, const int32_t* ik, const int64_t* qoff,
                            const double* Eab, int64_t sEab, const double* Ecd, int64_t sEcd, const double* PQ,
                            int64_t sPQ, double* Tm, int64_t sT, double* out, const double** a1, const double** b1,
                            double** c1, const double** a2, const double** b2, double** c2, cudaStream_t s);

// Schwarz reduction: Q[p] = sqrt(max_ab |diag of shellset p|).
cudaError_t launch_schwarz_reduce(const int64_t* off, const int32_t* nab, int64_t n, const double* vals,
                                  double* Q, cudaStream_t s);

}  // namespace mdx
