// Launch geometry of the pipelined operator applications, as plain C++ (no
// CUDA) so that host code and a CPU-side test share one definition: rows per
// tile, whether x0 rides in the bulk copies, stage sizes and counts.  Every
// bulk copy (TMA) source, destination and size must be a multiple of 16
// bytes; these functions choose only geometries that keep it so.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define DFM_GEOM_HD __host__ __device__
#else
#define DFM_GEOM_HD
#endif

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

// ---- bases above N_p = 8 (wide.cu): N_b = 55 .. 231 ----
constexpr int kNarrowMaxNb = 45;  // largest basis of the per-warp kernels (N_p = 8)
constexpr int kWideMaxNp = 20;    // largest order of the wide kernels (N_b = 231)

// Assembly of one face pair by one block per tile of test rows: the block's
// CG x RG threads each own 8 test rows x 8 trial columns of the tile (CG =
// NS NBP / 8 column groups, RG row groups, TRW = 8 RG rows per tile), NC nodes
// are staged per pass (Z(p) of the NBP padded Zernike columns, and for each
// of the NS source spatial functions the weighted w Z(p') of the tile's
// rows), evaluated by threads [0, NC) and [NC, 2 NC).  NS = 1: the
// piecewise-constant spatial basis (block side NB); NS = 3: the linear one
// (block side 3 NB, columns padded to NBP per spatial function).
struct WideAsm {
  int nb, nbp;   // Zernike functions per face and their padding to 8
  int ns, nrow;  // spatial functions per face, block side ns nb
  int cg, rg;    // column and row groups of a tile
  int trw;       // test rows per tile (8 rg)
  int ntile;     // tiles per face pair
  int threads;   // block size (a multiple of 32, >= cg rg and >= 2 nc)
  int nc;        // nodes staged per pass
  int ldq, ldp;  // staging row strides (floats): trw + 4, nbp + 4
  int64_t smem;  // dynamic shared memory bytes beyond the patch state
};

inline WideAsm wide_asm_geometry(int nb, int ns = 1) {
  WideAsm g{};
  g.nb = nb;
  g.nbp = (nb + 7) / 8 * 8;
  g.ns = ns;
  g.nrow = ns * nb;
  g.cg = ns * g.nbp / 8;
  const int nrg = (g.nrow + 7) / 8;  // row groups of the whole block
  int max_rg = 256 / g.cg;
  if (max_rg < 1) max_rg = 1;
  g.ntile = (nrg + max_rg - 1) / max_rg;
  g.rg = (nrg + g.ntile - 1) / g.ntile;
  g.trw = 8 * g.rg;
  g.threads = (g.cg * g.rg + 31) / 32 * 32;
  if (g.threads < 64) g.threads = 64;
  g.nc = g.threads / 2 < 64 ? g.threads / 2 : 64;
  g.ldq = g.trw + 4;
  g.ldp = g.nbp + 4;
  g.smem = (int64_t)g.nc * (ns * g.ldq + g.ldp) * 4 + ((int64_t)g.trw + 2 * 32) * 4;
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
// kHopTileBytes, else one pass
constexpr int hop_tile_rows(int nb, int eb, bool scaled) {
  const int step = (32 * kHopConsumerWarps) / hop_nbp(nb);
  const int two = step * kHopPasses < 32 ? step * kHopPasses : 32;
  return (two * hop_row_bytes(nb, eb, scaled) <= kHopTileBytes) ? two : (step < 32 ? step : 32);
}

// staged bytes per tile row for R right-hand sides: the copy row, each right-hand
// side's source-tet coefficients (4 NBP vector entries) and its x0 row (NBP entries)
constexpr int64_t hop_stage_bytes(int nb, int eb, bool scaled, int vb, int R) {
  return hop_tile_rows(nb, eb, scaled) *
         (hop_row_bytes(nb, eb, scaled) + (int64_t)R * (4 * hop_nbp(nb) * vb + hop_nbp(nb) * vb));
}

// right-hand sides per launch: at most kHopMaxRhs, and few enough that two
// stages fit (0 when even one does not)
inline int hop_rhs_chunk(int nb, int eb, bool scaled, int vb) {
  int r = kHopMaxRhs;
  while (r > 0 && 2 * hop_stage_bytes(nb, eb, scaled, vb, r) > kStageBudget) --r;
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

// ---- tensor-core hops on the fragment-ordered copy (hop_frag_kernel) ----
constexpr int kFragGroups = 2;          // consumer groups taking alternate tiles
constexpr int kFragGroupWarps = 4;      // warps per consumer group
constexpr int kFragMaxStages = 8;
constexpr int kFragGroupMin = 4;        // right-hand sides from which vectors are grouped by 8
constexpr int64_t kFragStageTarget = 48 * 1024;  // default stage size

// the fragment-ordered copy serves bases whose padded width is a multiple of 16
constexpr bool frag_basis(int nb) { return hop_nbp(nb) % 16 == 0; }
// bytes of one face row of one hop-vector group (w = 1 or 8 right-hand sides, FP16)
constexpr int64_t frag_xrow_bytes(int nb, int w) { return (int64_t)hop_nbp(nb) * w * 2; }
// staged bytes of one tile row: the copy row, per group the gathered source
// rows (4 slots) and the x0 row
constexpr int64_t frag_row_stage_bytes(int nb, int eb, bool scaled, int w, int rgl) {
  return hop_row_bytes(nb, eb, scaled) + (int64_t)rgl * 5 * frag_xrow_bytes(nb, w);
}

struct Frag {
  int rpt;              // operator rows per tile (<= 32)
  int stages;           // pipeline stages (<= kFragMaxStages)
  int64_t stage_bytes;  // bytes of one stage
};

// Tile rows and stages: rpt_req / stages_req if given (clamped to what fits),
// else tiles of about kFragStageTarget bytes whose (row, group) items split
// evenly over a consumer group's warps, and as many stages as fit.
inline Frag frag_geometry(int nb, int eb, bool scaled, int w, int rgl, int rpt_req = 0, int stages_req = 0) {
  const int64_t row = frag_row_stage_bytes(nb, eb, scaled, w, rgl);
  int rpt = rpt_req > 0 ? rpt_req : (int)(kFragStageTarget / row);
  if (rpt > 32) rpt = 32;
  if (rpt_req <= 0) {
    const int unit = rgl >= kFragGroupWarps ? 1 : kFragGroupWarps / rgl;  // rows per full round of the group
    if (rpt >= unit) rpt -= rpt % unit;
  }
  if (rpt < 1) rpt = 1;
  while (rpt > 1 && 2 * rpt * row > kStageBudget) --rpt;  // at least two stages
  Frag g{};
  g.rpt = rpt;
  g.stage_bytes = rpt * row;
  int64_t st = kStageBudget / g.stage_bytes;
  if (st > kFragMaxStages) st = kFragMaxStages;
  if (stages_req > 0 && stages_req < st) st = stages_req;
  // a multiple of the consumer groups: tile i and tile i - stages, the last
  // user of its stage, then belong to the same group, which has consumed it
  // (its barrier phase completed) before it waits for tile i; with another
  // count a group could meet the stage's barrier a phase behind and read the
  // parity of an older phase as complete
  st -= st % kFragGroups;
  g.stages = (int)st;
  return g;
}

// (block k, test a, trial b) of value e of one row of the fragment-ordered
// copy (hop_frag.cuh): per block, 16 x 16 tiles in (m-tile, k-tile) order,
// each holding lane (g, t)'s values (row g; columns 2t, 2t+1, 2t+8, 2t+9) for
// the 32 lanes, then those of row g + 8 for the lanes with g + 8 < vm, the
// tile's rows (vm = min(16, nb - 16 m-tile)); b >= nb are pads
struct FragPos {
  int k, a, b;
};
DFM_GEOM_HD inline FragPos frag_pos(int64_t e, int nb, int nbp) {
  FragPos p;
  p.k = (int)(e / ((int64_t)nb * nbp));
  int rem = (int)(e - (int64_t)p.k * nb * nbp);
  const int mt = rem / (16 * nbp);
  rem -= mt * 16 * nbp;
  const int vm = nb - 16 * mt < 16 ? nb - 16 * mt : 16;
  const int kt = rem / (16 * vm);
  rem -= kt * 16 * vm;
  const int half = rem < 128 ? 0 : 8;
  const int idx = rem < 128 ? rem : rem - 128;
  const int lane = idx >> 2, j = idx & 3;
  p.a = 16 * mt + half + (lane >> 2);
  p.b = 16 * kt + 2 * (lane & 3) + (j & 1) + (j >= 2 ? 8 : 0);
  return p;
}

// dynamic shared memory of a launch: barriers, the per-stage row map, stages
inline int64_t frag_smem_bytes(const Frag& g) {
  return 128 + ((int64_t)kFragMaxStages * 32 * 4 + 127) / 128 * 128 + (int64_t)g.stages * g.stage_bytes;
}

}  // namespace geom
}  // namespace dfm
