// Launch geometry of the pipelined operator applications, as plain C++ (no
// CUDA) so that host code and a CPU-side test share one definition: rows per
// tile, whether x0 rides in the bulk copies, stage sizes and counts.  Every
// bulk copy (TMA) source, destination and size must be a multiple of 16
// bytes; these functions choose only geometries that keep it so.
#pragma once

#include <stdint.h>

namespace dfm {
namespace geom {

constexpr int64_t kStageBudget = 200 * 1024 - 1024;  // dynamic shared memory per block for the stages

// row stride of the block storage (elements): 3 N_b^2 rounded up to 8
constexpr int64_t op_row_stride(int nb) { return ((3 * (int64_t)nb * nb + 7) / 8) * 8; }

// ---- forward application y = x0 + alpha sum_k coef_k B_k x (spmv_tma_kernel) ----
struct Fwd {
  int rpt;            // operator rows per tile
  int stage_x0;       // 1: x0 slices are staged by bulk copies (else read directly)
  int stages;         // pipeline stages (0: a row does not fit)
  int64_t row_bytes;  // staged bytes per operator row (all right-hand sides)
};

// nb basis functions, tv / tx bytes per block entry / vector entry, K
// operators, R right-hand sides (<= 16) staged per pass, nrows operator rows;
// x0_ptr_aligned: x0 given and 16-byte aligned; max_stages: the kernel's stage
// count.
inline Fwd fwd_geometry(int nb, int tv, int tx, int K, int R, int64_t nrows, bool x0_ptr_aligned, int max_stages) {
  Fwd g{};
  int rpt = 128 / nb;
  if (rpt < 1) rpt = 1;
  if (rpt > 32) rpt = 32;
  const int64_t x0_row = (int64_t)nb * tx;
  // x0 rides in the pipeline when every tile's slice (rows R0 .. R0 + rpt of
  // every right-hand side) starts on a 16-byte boundary in global and shared memory
  auto x0_aligned = [&](int rp) -> int {
    return (x0_ptr_aligned && (x0_row % 16 == 0 || ((nrows % rp) == 0 && (rp * x0_row) % 16 == 0))) ? 1 : 0;
  };
  int sx = x0_aligned(rpt);
  auto bytes_per_row = [&]() -> int64_t {
    return K * op_row_stride(nb) * tv + (int64_t)R * 4 * nb * tx + (sx ? (int64_t)R * x0_row : 0);
  };
  int64_t rb = bytes_per_row();
  while (rpt > 1 && rpt * rb * 2 > kStageBudget) --rpt;  // keep at least two stages
  if (sx && !x0_aligned(rpt)) {  // smaller tiles break the slice alignment: read x0 directly
    sx = 0;
    rb = bytes_per_row();
  }
  int64_t st = kStageBudget / (rpt * rb);
  if (st > max_stages) st = max_stages;
  g.rpt = rpt;
  g.stage_x0 = sx;
  g.stages = (int)st;
  g.row_bytes = rb;
  return g;
}

// ---- preconditioner hops on the low-precision copy (hop_kernel) ----
constexpr int kHopConsumerWarps = 8;
constexpr int kHopPasses = 2;  // consumer passes per tile when the copy rows are small
constexpr int kHopMaxRhs = 16;               // right-hand sides staged per pass
constexpr int64_t kHopTileBytes = 48 * 1024;  // copy bytes of a tile for two consumer passes
constexpr int64_t kHopTwoBlockBytes = 110 * 1024;  // stage bytes that still fit two blocks per SM

constexpr int hop_nbp(int nb) { return (nb + 7) / 8 * 8; }

// bytes of one row of the copy: the values (eb bytes each, padded to 16) and,
// for a scaled format, a 16-byte field holding the row's scale
constexpr int64_t hop_body_bytes(int nb, int eb) { return (3 * (int64_t)nb * hop_nbp(nb) * eb + 15) / 16 * 16; }
constexpr int64_t hop_row_bytes(int nb, int eb, bool scaled) { return hop_body_bytes(nb, eb) + (scaled ? 16 : 0); }

// rows per tile: two consumer passes of (32 x consumer warps) / NBP rows (at
// most 32, one per producer lane) when the tile's copy rows stay within
// kHopTileBytes, else one pass; the tensor-core consumer (several right-hand
// sides, whose staged coefficients already fill the tile) always takes one
constexpr int hop_tile_rows(int nb, int eb, bool scaled, bool mma) {
  const int step = (32 * kHopConsumerWarps) / hop_nbp(nb);
  const int two = step * kHopPasses < 32 ? step * kHopPasses : 32;
  return (!mma && two * hop_row_bytes(nb, eb, scaled) <= kHopTileBytes) ? two : (step < 32 ? step : 32);
}

// staged bytes per tile row for R right-hand sides: the copy row, each right-hand
// side's source-tet coefficients (4 NBP vector entries, plus a 16-byte gap
// for the tensor-core consumer) and its x0 row (NBP entries)
constexpr int64_t hop_stage_bytes(int nb, int eb, bool scaled, int vb, int R, bool mma) {
  return hop_tile_rows(nb, eb, scaled, mma) *
         (hop_row_bytes(nb, eb, scaled) + (int64_t)R * (4 * hop_nbp(nb) * vb + (mma ? 16 : 0) + hop_nbp(nb) * vb));
}

// right-hand sides per launch: at most kHopMaxRhs, and few enough that two
// stages fit (0 when even one does not)
inline int hop_rhs_chunk(int nb, int eb, bool scaled, int vb, bool mma) {
  int r = kHopMaxRhs;
  while (r > 0 && 2 * hop_stage_bytes(nb, eb, scaled, vb, r, mma) > kStageBudget) --r;
  return r;
}

// stages for a tile of stage_bytes: up to max_stages, but no more than leave
// room for two blocks per SM when the tiles are large
inline int hop_stages(int64_t stage_bytes, int max_stages) {
  int64_t s = kStageBudget / stage_bytes;
  if (s > max_stages) s = max_stages;
  if (s > 2 && s * stage_bytes > kHopTwoBlockBytes) s = kHopTwoBlockBytes / stage_bytes < 2 ? 2 : kHopTwoBlockBytes / stage_bytes;
  return (int)s;
}

}  // namespace geom
}  // namespace dfm
