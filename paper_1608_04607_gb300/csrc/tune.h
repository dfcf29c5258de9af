// Autotuner of launch geometries (tile rows and pipeline stages) for the
// pipelined kernels: the first launch of a kernel for a given shape times
// every candidate geometry on the caller's own arguments (each candidate
// writes the same output, so the last launch, with the fastest geometry,
// leaves the right result), keeps the fastest, and later launches of that
// shape use it.  Geometry changes no arithmetic: outputs are identical.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <vector>

namespace dfm {
namespace tune {

struct Key {
  int kind;       // which kernel family
  int nb, prec;   // basis size, copy precision
  int w, rgl;     // right-hand sides per group, groups per launch
  int trans;
  int64_t nrows;  // problem size
  int device;
};

struct Geometry {
  int rpt, stages;
  float ms;  // mean time of the timed launches (0: not timed)
};

// The geometry for key: the cached choice, else (tuning on, stream not being
// captured) the fastest of `cands` timed with `launch`, else `fallback`.
// launch(rpt, stages) enqueues one launch on st and returns a DFM status.
int choose(const Key& key, cudaStream_t st, const std::vector<Geometry>& cands, const Geometry& fallback,
           const std::function<int(int, int)>& launch, Geometry* out);

}  // namespace tune
}  // namespace dfm
