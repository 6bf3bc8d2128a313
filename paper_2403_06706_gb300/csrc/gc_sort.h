// gc_sort.h -- cell sort of the particle arrays (gather locality; no effect on results).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gc_internal.h"

namespace gcp {

// Scratch of the sort, owned by the context: the alternate state arrays (the sorted copy
// is written there and the pointers are swapped), per-particle keys and ranks, and the
// bin counts / offsets.
struct SortWork {
    StateDev alt{};
    int64_t cap = 0;
    uint32_t *key = nullptr, *rank = nullptr, *hist = nullptr;
    int64_t nbins_cap = 0;
};

// Counting sort of st by coarse grid cell (cells merged by a power of two until at most
// 2^18 bins remain). Swaps st's arrays with the sorted copy in w.alt.
cudaError_t sort_by_cell(SortWork &w, StateDev &st, const GridHost &g, int n_ens, cudaStream_t s);
// Copy st into w.alt in id order: slot id - id_lo (ids must be a permutation of
// [id_lo, id_lo + n)). Used to return the state in id order after cell sorts.
cudaError_t unpermute_to_alt(SortWork &w, const StateDev &st, uint32_t id_lo, cudaStream_t s);
void sort_free(SortWork &w);
// Allocate the sort's buffers for st and grid g now (before a graph capture, which cannot
// allocate).
cudaError_t sort_reserve(SortWork &w, const StateDev &st, const GridHost &g);
// load the sort kernels now (see preload_kernels)
cudaError_t sort_preload();
// A full set of state arrays of capacity cap (F0/F1 as [4][cap]) and its release.
cudaError_t alloc_state(StateDev &s, int64_t cap);
void free_state_arrays(StateDev &s);
// kernels launched by one sort_by_cell / unpermute_to_alt call
constexpr int kSortKernels = 3;
constexpr int kUnpermuteKernels = 1;

} // namespace gcp
