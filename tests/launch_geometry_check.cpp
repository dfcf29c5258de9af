// Host-side check of the launch geometry of the pipelined operator
// applications (launch_geometry.h): for every basis size, precision, number of
// combined operators (up to 4, FP32 only) and right-hand sides and a set of
// row counts, every bulk
// copy starts and ends on a 16-byte boundary, shared memory stays within a
// block's 227 KB, a tile has at most 32 rows and at least the required stages.
// Built and run by tests/test_launch_geometry.py; prints "ok" or the first
// violation and exits non-zero.
#include <cstdio>
#include <initializer_list>

#include "launch_geometry.h"

using namespace dfm::geom;

static int fail(const char* what, int nb, int a, int b, int c, long long d) {
  std::printf("violation: %s (nb=%d, %d, %d, %d, %lld)\n", what, nb, a, b, c, d);
  return 1;
}

int main() {
  const int nbs[] = {1, 3, 6, 10, 15, 21, 28, 36, 45};
  const long long rows[] = {4, 24, 28, 644, 648, 4 * 6001, 192000, 648000, 786432};
  const long long kSmem = 227 * 1024;
  long long checked = 0;
  // forward application: block bytes tv, vector bytes tx, K operators, R right-hand sides
  for (int nb : nbs)
    for (int tv : {2, 4, 8})
      for (int tx : {4, 8})
        for (int K = 1; K <= (tv == 4 ? 4 : 1); ++K)  // combined operators are FP32
          for (int R = 1; R <= 16; ++R)
            for (long long nrows : rows)
              for (int x0a = 0; x0a < 2; ++x0a) {
                const Fwd g = fwd_geometry(nb, tv, tx, K, R, nrows, x0a != 0, 4);
                if (g.rpt < 1 || g.rpt > 32) return fail("rows per tile", nb, tv, tx, R, g.rpt);
                if (g.stages < 1) return fail("no stage fits", nb, tv, tx, R, g.row_bytes);
                const long long stride = op_row_stride(nb) * tv;
                if (stride % 16) return fail("row stride", nb, tv, tx, R, stride);
                const long long xblk = 4LL * nb * tx;
                if (xblk % 16) return fail("x block", nb, tv, tx, R, xblk);
                const long long x0row = (long long)nb * tx;
                const long long x0b = g.stage_x0 ? (long long)R * g.rpt * x0row : 0;
                const long long stage = K * g.rpt * stride + (long long)R * g.rpt * xblk + (x0b + 15) / 16 * 16;
                const long long smem = 128 + ((long long)g.stages * g.rpt * 4 + 127) / 128 * 128 +
                                       (long long)g.stages * (g.rpt * g.row_bytes + 16);
                if (smem > kSmem) return fail("shared memory", nb, tv, tx, R, smem);
                if (stage % 16 || stage > g.rpt * g.row_bytes + 16) return fail("stage size", nb, tv, tx, R, stage);
                if (g.stage_x0) {
                  if (!x0a) return fail("x0 staged without an aligned pointer", nb, tv, tx, R, 0);
                  const long long ntiles = (nrows + g.rpt - 1) / g.rpt;
                  for (long long ti = 0; ti < ntiles; ti = (ti == 4096 && ntiles > 4097) ? ntiles - 1 : ti + 1) {
                    const long long R0 = ti * g.rpt;  // the first 4097 tiles and the last (ragged) one
                    const long long nr = nrows - R0 < g.rpt ? nrows - R0 : g.rpt;
                    for (int rhs = 0; rhs < R; ++rhs) {
                      ++checked;
                      if (((rhs * nrows + R0) * x0row) % 16) return fail("x0 source", nb, tv, tx, R, R0);
                      if ((nr * x0row) % 16) return fail("x0 size", nb, tv, tx, R, R0);
                      const long long dst = K * g.rpt * stride + (long long)R * g.rpt * xblk + rhs * g.rpt * x0row;
                      if (dst % 16) return fail("x0 destination", nb, tv, tx, R, R0);
                    }
                  }
                }
              }
  // preconditioner hops (CUDA-core kernel): copy bytes per value eb (FP16/BF16: 2,
  // e4m3: 1 with a row scale), vector bytes vb (FP16: 2, FP32: 4)
  struct Fmt {
    int eb;
    bool scaled;
    int vb;
  };
  const Fmt fmts[] = {{2, false, 2}, {2, false, 4}, {1, true, 2}};
  for (int nb : nbs)
    for (const Fmt& f : fmts) {
      const int rpt = hop_tile_rows(nb, f.eb, f.scaled);
      const int step = (32 * kHopConsumerWarps) / hop_nbp(nb);
      if (rpt < 1 || rpt > 32 || (rpt != step && rpt != 2 * step)) return fail("hop rows per tile", nb, f.eb, f.vb, 0, rpt);
      const long long row = hop_row_bytes(nb, f.eb, f.scaled);
      if (row % 16) return fail("hop copy row", nb, f.eb, f.vb, 0, row);
      const long long xblk = 4LL * hop_nbp(nb) * f.vb, x0row = (long long)hop_nbp(nb) * f.vb;
      if (xblk % 16 || x0row % 16) return fail("hop vector rows", nb, f.eb, f.vb, 0, xblk);
      const int chunk = hop_rhs_chunk(nb, f.eb, f.scaled, f.vb);
      if (chunk < 1) return fail("hop right-hand-side chunk", nb, f.eb, f.vb, 0, chunk);
      for (int R = 1; R <= chunk; ++R) {
        ++checked;
        const long long stage = hop_stage_bytes(nb, f.eb, f.scaled, f.vb, R);
        if (stage != rpt * row + (long long)R * rpt * (xblk + x0row)) return fail("hop stage bytes", nb, f.eb, f.vb, R, stage);
        const int stages = hop_stages(stage, 2);
        if (stages < 2) return fail("hop stages", nb, f.eb, f.vb, R, stage);
        const long long smem = 128 + (2LL * rpt * 4 + 127) / 128 * 128 + (long long)stages * stage;
        if (smem > kSmem) return fail("hop shared memory", nb, f.eb, f.vb, R, smem);
      }
    }
  // tensor-core hops on the fragment-ordered copy: every bulk copy (copy rows,
  // x0 slices, gathered face rows) 16-byte aligned and sized, shared memory
  // within a block, stages >= 2, for the default and requested geometries
  for (int nb : nbs) {
    if (!frag_basis(nb)) continue;
    const int nbp = hop_nbp(nb);
    // the layout: every (block, test < nb, trial < nbp) exactly once, and the
    // offsets the consumer loads give the mma.sync A-fragment entries
    static int seen[3 * 48 * 48];
    for (int i = 0; i < 3 * nb * nbp; ++i) seen[i] = 0;
    for (long long e = 0; e < 3LL * nb * nbp; ++e) {
      const FragPos p = frag_pos(e, nb, nbp);
      if (p.k < 0 || p.k > 2 || p.a < 0 || p.a >= nb || p.b < 0 || p.b >= nbp) return fail("frag position", nb, p.k, p.a, p.b, e);
      ++seen[(p.k * nb + p.a) * nbp + p.b];
    }
    for (int i = 0; i < 3 * nb * nbp; ++i)
      if (seen[i] != 1) return fail("frag layout not a bijection", nb, i, seen[i], 0, 0);
    for (int k = 0; k < 3; ++k)
      for (int mt = 0; mt < nbp / 16; ++mt)
        for (int kt = 0; kt < nbp / 16; ++kt)
          for (int lane = 0; lane < 32; ++lane)
            for (int half = 0; half < 2; ++half)
              for (int j = 0; j < 4; ++j) {
                const int vm = nb - 16 * mt < 16 ? nb - 16 * mt : 16;
                const int g = lane >> 2, t = lane & 3;
                if (half && g + 8 >= vm) continue;  // rows past nb are not stored (the consumer loads 0)
                const long long e = (long long)k * nb * nbp + 16LL * mt * nbp + (long long)kt * 16 * vm +
                                    (half ? 128 : 0) + lane * 4 + j;
                const FragPos p = frag_pos(e, nb, nbp);
                const int want_a = 16 * mt + g + 8 * half;
                const int want_b = 16 * kt + 2 * t + (j & 1) + (j >= 2 ? 8 : 0);
                ++checked;
                if (p.k != k || p.a != want_a || p.b != want_b) return fail("frag fragment entry", nb, mt, kt, lane, e);
              }
    for (const Fmt& f : fmts) {
      if (f.vb != 2) continue;  // FP16 hop vectors only
      for (int w : {1, 8})
        for (int rgl = 1; rgl <= (w == 8 ? 2 : 1); ++rgl)
          for (int rpt_req : {0, 1, 2, 3, 4, 6, 8, 12, 16, 24, 32})
            for (int st_req : {0, 2, 3, 4, 6, 8}) {
              const Frag g = frag_geometry(nb, f.eb, f.scaled, w, rgl, rpt_req, st_req);
              ++checked;
              if (g.rpt < 1 || g.rpt > 32) return fail("frag rows per tile", nb, f.eb, w, rgl, g.rpt);
              if (g.stages < 2 || g.stages > kFragMaxStages || g.stages % kFragGroups)
                return fail("frag stages", nb, f.eb, w, rgl, g.stages);
              if (frag_smem_bytes(g) > kSmem) return fail("frag shared memory", nb, f.eb, w, rgl, frag_smem_bytes(g));
              const long long row = hop_row_bytes(nb, f.eb, f.scaled), xr = frag_xrow_bytes(nb, w);
              const long long x_off = g.rpt * row, x0_off = x_off + (long long)g.rpt * rgl * 4 * xr;
              if (row % 16 || xr % 16 || x_off % 16 || x0_off % 16 || g.stage_bytes % 16 ||
                  g.stage_bytes != x0_off + (long long)rgl * g.rpt * xr)
                return fail("frag stage layout", nb, f.eb, w, rgl, g.stage_bytes);
              if (rpt_req == 0 && g.stage_bytes > kFragStageTarget && g.rpt > 1)
                return fail("frag default tile", nb, f.eb, w, rgl, g.stage_bytes);
            }
    }
  }
  // wide assembly (N_p = 9..20 with one spatial function, 0..8 with the three
  // of the linear basis): tiles cover the block once, thread roles fit the
  // block, staged rows hold every read of the accumulation (rows 8 rg ..
  // 8 rg + 7 of a tile; columns 4 cg .. 4 cg + 3 and NS NBP/2 + 4 cg .., each
  // group inside one spatial function's NBP columns) as aligned 16-byte
  // vectors, and two blocks fit an SM's shared memory
  for (int ns : {1, 3})
    for (int np = (ns == 1 ? 9 : 0); np <= (ns == 1 ? kWideMaxNp : 8); ++np) {
      const int nb = (np + 1) * (np + 2) / 2;
      const WideAsm g = wide_asm_geometry(nb, ns);
      ++checked;
      if (g.threads % 32 || g.threads > 256 || g.threads < 64) return fail("wide threads", nb, g.threads, ns, 0, 0);
      if (g.cg * g.rg > g.threads || 2 * g.nc > g.threads || g.nc < 1 || g.nc > 64)
        return fail("wide roles", nb, g.cg, g.rg, g.nc, g.threads);
      if (g.nbp < nb || g.nbp % 8 || g.cg * 8 != ns * g.nbp || g.nrow != ns * nb)
        return fail("wide columns", nb, g.nbp, g.cg, ns, 0);
      if ((long long)g.trw * g.ntile < g.nrow || (long long)g.trw * (g.ntile - 1) >= g.nrow)
        return fail("wide tiles", nb, g.trw, g.ntile, ns, 0);
      if (g.trw != 8 * g.rg || g.ldq != g.trw + 4 || g.ldp != g.nbp + 4 || g.ldq % 4 || g.ldp % 4 ||
          (ns * g.nbp / 2) % 4)
        return fail("wide strides", nb, g.ldq, g.ldp, g.trw, ns);
      if (8 * (g.rg - 1) + 7 >= g.ldq) return fail("wide staged rows", nb, g.rg, g.cg, ns, 0);
      for (int cg = 0; cg < g.cg; ++cg)
        for (int c : {4 * cg, ns * g.nbp / 2 + 4 * cg}) {
          const int a = c / g.nbp, j = c - a * g.nbp;
          if (a < 0 || a >= ns || j % 4 || j + 3 >= g.nbp) return fail("wide column group", nb, cg, c, ns, 0);
        }
      if ((g.nc * (long long)g.ldq * 4) % 16) return fail("wide zq plane", nb, g.nc, g.ldq, ns, 0);
      const long long static_smem = 4096;  // patch state and pair constants
      if (2 * (g.smem + static_smem) > 228LL * 1024 || g.smem > 200 * 1024)
        return fail("wide shared memory", nb, ns, 0, 0, g.smem);
      if (ns == 1) {  // the same geometry as before the spatial functions were added
        const WideAsm h = wide_asm_geometry(nb);
        if (h.cg != g.cg || h.trw != g.trw || h.threads != g.threads || h.smem != g.smem)
          return fail("wide default", nb, 0, 0, 0, 0);
      }
    }
  std::printf("ok %lld\n", checked);
  return 0;
}
