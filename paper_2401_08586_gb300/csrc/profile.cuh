// profile.cuh -- launch counting and per-kernel event timing (profile.cu).
#pragma once

#include <cuda_runtime.h>
#include <string.h>

namespace sph {

enum ProfTag {
    TAG_BOUNDS,
    TAG_HASH,
    TAG_SCAN,
    TAG_SCATTER,
    TAG_SORT,
    TAG_CONVERT,
    TAG_COUNT,
    TAG_FILL,
    TAG_DENSITY,
    TAG_CANON,
    TAG_FUSED,
    TAG_BATCH,
    TAG_STEP,
    TAG_COUNT_
};

// Add k to the number of kernels the library has launched.
void note_launch(int k);
long long launch_count();
const char *tag_name(int tag);

// While profiling is enabled, records a CUDA event on `s` at construction and
// another at destruction; the elapsed time is credited to `tag`.
class ProfScope {
   public:
    ProfScope(int tag, cudaStream_t s);
    ~ProfScope();

   private:
    int tag_;
    cudaStream_t s_;
    void *a_;
};

void prof_enable(int on);
// While a thread records a CUDA graph its ProfScopes record nothing (event
// timing does not apply to captured work).
void prof_set_capturing(bool on);
// Enable timing for a comma-separated list of tag names only (NULL: all);
// -1 if a name is unknown (nothing changed).
int prof_select(const char *names);
// Measured FP64 FMA throughput of the current device, in FLOP/s (2 per FMA).
int fp64_fma_rate(double *flops);
void prof_reset();
int prof_read(const char *name, double *ms, long long *calls);

}  // namespace sph
