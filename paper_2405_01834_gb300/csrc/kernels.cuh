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
  const uint32_t* hdec;      // Hermite index decode table
  const int32_t* hdec_off;   // start of each total order N in hdec
  double* out;
  int* err;
};

cudaError_t launch_quartets(const QuartetLaunch& a, cudaStream_t s);
cudaError_t kernel_attributes_init();

// Schwarz reduction: Q[p] = sqrt(max_ab |diag of shellset p|).
cudaError_t launch_schwarz_reduce(const int64_t* off, const int32_t* nab, int64_t n, const double* vals,
                                  double* Q, cudaStream_t s);

}  // namespace mdx
