// Many layers' ELT folds (Algorithm 1, steps 1-3, per catalog event) in one
// launch, for pricing plans that re-fold a fixed list of layers every step.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "ara_internal.cuh"

namespace ara {

// One layer's fold in a batch: its ELT list, occurrence terms, fixed-point
// exponent and output table/bitmap (as for launch_fold); fp32 selects the
// binary32 combine of FP32-table layers.  stride > 1 writes the layer's
// entries into an interleaved table of stride layers (table points at this
// layer's first entry; event e's entry is table[e * stride]), and several
// jobs may share one bitmap, which then receives the union of their bits.
struct FoldJob {
  const EltDesc *elts;
  int32_t n_elts;
  int32_t q;
  double occ_ret, occ_lim;
  void *table;
  uint32_t *bitmap;
  uint32_t bm_mul;
  int32_t fp32;
  int32_t stride;
};

// Clear the bitmaps (words 32-bit words each) and sentinel entries of n_jobs
// layers, then fold them all in one launch; max_elts = the largest n_elts.
// d_jobs is device memory that stays valid while the launches run.
cudaError_t launch_fold_batch(const FoldJob *d_jobs, int n_jobs, int max_elts, int32_t catalog, int32_t words,
                              cudaStream_t s);

}  // namespace ara
