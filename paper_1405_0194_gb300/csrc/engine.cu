// C ABI of the plan: host symbolic analysis + upload (pexsi_setup), and the
// batched numeric drivers (pole batches through assembly, factorisation,
// selected inversion and the pole sum; inertia shift batches).
#include <algorithm>
#include <cfloat>
#include <cstdio>
#include <climits>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "plan.hpp"

namespace pexsi {

// ------------------------------------------------------------------ profiler
namespace {
const char* const kProfNames[PEXSI_PROFILE_CLASSES] = {
    "assemble", "extend_add", "diag_inv", "panel_solve", "schur_update", "gather",
    "selinv_offdiag", "selinv_diag_partial", "selinv_diag_reduce", "pole_sum", "trace", "split_slice"};
}

cudaEvent_t Profiler::begin(cudaStream_t st) {
  if (!on) return nullptr;
  cudaEvent_t a;
  if (!pool.empty()) { a = pool.back(); pool.pop_back(); }
  else ck(cudaEventCreate(&a), "cudaEventCreate(profile)");
  ck(cudaEventRecord(a, st), "cudaEventRecord(profile)");
  return a;
}

void Profiler::end(cudaEvent_t a, int cls, cudaStream_t st, double fl, double by, int kernels, double tensor_fl) {
  if (!on || !a) return;
  cudaEvent_t b;
  if (!pool.empty()) { b = pool.back(); pool.pop_back(); }
  else ck(cudaEventCreate(&b), "cudaEventCreate(profile)");
  ck(cudaEventRecord(b, st), "cudaEventRecord(profile)");
  pending.push_back({cls, a, b, fl, by, kernels, tensor_fl});
}

void Profiler::drain() {
  for (auto& q : pending) {
    ck(cudaEventSynchronize(q.b), "cudaEventSynchronize(profile)");
    float t = 0;
    ck(cudaEventElapsedTime(&t, q.a, q.b), "cudaEventElapsedTime(profile)");
    launches[q.cls] += q.kernels;
    ms[q.cls] += t;
    flops[q.cls] += q.flops;
    bytes[q.cls] += q.bytes;
    tensor[q.cls] += q.tensor;
    pool.push_back(q.a);
    pool.push_back(q.b);
  }
  pending.clear();
}

void Profiler::reset() {
  drain();
  for (int c = 0; c < PEXSI_PROFILE_CLASSES; ++c) { launches[c] = 0; ms[c] = flops[c] = bytes[c] = tensor[c] = 0; }
}

void Profiler::destroy() {
  for (auto& q : pending) { cudaEventDestroy(q.a); cudaEventDestroy(q.b); }
  for (auto e : pool) cudaEventDestroy(e);
  pending.clear();
  pool.clear();
}

// ------------------------------------------------------------------ workspaces
// Split-K partials of the FP64 Takahashi step, per batch member: kMaxKsplit
// tiles of kTile x b for each 64-row tile slot of the partial layout.
int64_t kpart_stride(const pexsi_plan* p) {
  return p->oz_slices > 0 ? 0 : p->part_stride / (int64_t(p->b) * p->b) * kMaxKsplit * kTile * p->b;
}

int64_t bytes_per_pole(const pexsi_plan* p) {
  return (2 * p->sym.front_elems + p->part_stride + kpart_stride(p)) * int64_t(sizeof(double2)) +
         2 * p->sym.n * int64_t(p->b) * int64_t(sizeof(double)) +
         std::max(p->ozA_stride, 2 * p->ozA_stride_r) + std::max(p->ozB_stride, 2 * p->ozB_stride_r) +
         8 * (p->exA_stride + p->exB_stride) + 4 * p->ymax_stride;
}

int64_t bytes_fixed(const pexsi_plan* p) {
  return 9 * p->sym.nnz * int64_t(sizeof(double)) + 4 * p->trace_blocks * 8 + 4096;
}

namespace {
const int kBig = INT_MAX;
const unsigned long long kInfBits = 0x7FF0000000000000ull;
}  // namespace

// Clears the status words of one chain (0 = poles, 1 = inertia shifts): the
// first breakdown front, the smallest pivot ratio and the failure flag of
// the split-precision waits.
void reset_status(Workspace& ws, int which) {
  ck(cudaMemcpyAsync(ws.brk + which, &kBig, sizeof(int), cudaMemcpyHostToDevice, ws.stream), "status");
  ck(cudaMemcpyAsync(ws.minpiv + which, &kInfBits, sizeof(kInfBits), cudaMemcpyHostToDevice, ws.stream), "status");
  if (ws.ozfail) ck(cudaMemsetAsync(ws.ozfail + which, 0, sizeof(int), ws.stream), "status");
}

namespace {
template <typename T>
void wsalloc(T** ptr, size_t bytes, Workspace& ws, const char* what) {
  if (ws.async) ck(cudaMallocAsync(reinterpret_cast<void**>(ptr), bytes, ws.stream), what);
  else ck(cudaMalloc(reinterpret_cast<void**>(ptr), bytes), what);
  ws.bytes += int64_t(bytes);
}
}  // namespace

void workspace_alloc(const pexsi_plan* p, Workspace& ws, int batch, cudaStream_t stream, bool async) {
  ws.async = async;
  ws.stream = stream;
  ws.batch = batch;
  ws.bytes = 0;
  const size_t pool = size_t(p->sym.front_elems), nnz = size_t(p->sym.nnz);
  wsalloc(&ws.F, sizeof(double2) * pool * batch, ws, "alloc(F)");
  wsalloc(&ws.Y, sizeof(double2) * pool * batch, ws, "alloc(Y)");
  wsalloc(&ws.part, sizeof(double2) * size_t(p->part_stride) * batch, ws, "alloc(partials)");
  if (kpart_stride(p) > 0)
    wsalloc(&ws.kpart, sizeof(double2) * size_t(kpart_stride(p)) * batch, ws, "alloc(split-K partials)");
  wsalloc(&ws.H, sizeof(double) * nnz, ws, "alloc(H)");
  wsalloc(&ws.S, sizeof(double) * nnz, ws, "alloc(S)");
  wsalloc(&ws.out, sizeof(double) * nnz * 4, ws, "alloc(outputs)");
  // status words: [0] the pole chain (DM calls), [1] the inertia shifts
  // the inertia shifts' panel blocks before inversion: n x b per member, up to
  // 2 batch real members (or batch complex Hermitian ones)
  wsalloc(&ws.dsave, sizeof(double) * size_t(p->sym.n) * p->b * 2 * batch, ws, "alloc(inertia blocks)");
  wsalloc(&ws.brk, 2 * sizeof(int), ws, "alloc(status)");
  wsalloc(&ws.minpiv, 2 * sizeof(unsigned long long), ws, "alloc(status)");
  wsalloc(&ws.neg, sizeof(int) * kMaxBatch, ws, "alloc(status)");
  wsalloc(&ws.partials, sizeof(double) * 4 * p->trace_blocks, ws, "alloc(trace)");
  wsalloc(&ws.trace3, sizeof(double) * 4, ws, "alloc(trace)");
  if (p->oz_slices > 0) {
    // complex poles use `batch` members, the real inertia shifts up to 2 batch
    wsalloc(&ws.ozA, size_t(std::max(p->ozA_stride, 2 * p->ozA_stride_r)) * batch, ws, "alloc(split A)");
    wsalloc(&ws.ozB, size_t(std::max(p->ozB_stride, 2 * p->ozB_stride_r)) * batch, ws, "alloc(split B)");
    wsalloc(&ws.exA, sizeof(int) * size_t(p->exA_stride) * 2 * batch, ws, "alloc(split exponents)");
    wsalloc(&ws.exB, sizeof(int) * size_t(p->exB_stride) * 2 * batch, ws, "alloc(split exponents)");
    wsalloc(&ws.ozfail, 2 * sizeof(int), ws, "alloc(status)");
    wsalloc(&ws.ymax, sizeof(uint32_t) * size_t(p->ymax_stride) * batch, ws, "alloc(split row maxima)");
  }
  if (!ws.ev0) ck(cudaEventCreate(&ws.ev0), "cudaEventCreate");
  if (!ws.ev1) ck(cudaEventCreate(&ws.ev1), "cudaEventCreate");
  reset_status(ws, 0);
  reset_status(ws, 1);
}

void workspace_free(Workspace& ws) {
  void* ptrs[] = {ws.F,  ws.Y,        ws.part,  ws.H,    ws.S,   ws.out, ws.brk, ws.minpiv, ws.neg,
                  ws.partials, ws.trace3, ws.ainv, ws.ozA, ws.ozB, ws.exA, ws.exB, ws.ozfail, ws.ymax, ws.kpart,
                  ws.dsave};
  for (void* q : ptrs) {
    if (!q) continue;
    if (ws.async) cudaFreeAsync(q, ws.stream);
    else cudaFree(q);
  }
  if (ws.ev0) cudaEventDestroy(ws.ev0);
  if (ws.ev1) cudaEventDestroy(ws.ev1);
  for (Workspace::Graph& g : ws.graphs) cudaGraphExecDestroy(g.exec);
  if (ws.capture) cudaStreamDestroy(ws.capture);
  cudaStream_t st = ws.stream;
  bool async = ws.async;
  ws = Workspace();
  ws.stream = st;
  ws.async = async;
}

// ------------------------------------------------------------------ drivers
namespace {

struct PanelGeom {
  int nact = 0, row_tiles = 0, tri_tiles = 0, max_mp = 0, oz_schur = 0, oz_schur_r = 0;
  int oz_blk = 0, oz_blk_r = 0;  // split path: most tiles of the update of the rest of the panel block (cb > 0)
};

PanelGeom panel_geom(const Level& lv, int p0, int b, int cb = 0) {
  PanelGeom g;
  for (size_t t = 0; t < lv.fronts.size(); ++t) {
    if (lv.s[t] <= p0) break;
    ++g.nact;
    int bb = std::min(b, lv.s[t] - p0);
    int mp = lv.m[t] - p0 - bb;
    if (cb > 0) {
      const int cs = std::min(cb, lv.s[t]) - p0 - bb;
      g.oz_blk = std::max(g.oz_blk, oz_block_tiles(mp, cs, true));
      g.oz_blk_r = std::max(g.oz_blk_r, oz_block_tiles(mp, cs, false));
    }
    int rt = (mp + kTile - 1) / kTile;
    g.row_tiles = std::max(g.row_tiles, rt);
    g.tri_tiles = std::max(g.tri_tiles, rt * (rt + 1) / 2);
    g.max_mp = std::max(g.max_mp, mp);
    g.oz_schur = std::max(g.oz_schur, oz_schur_tiles(mp));
    g.oz_schur_r = std::max(g.oz_schur_r, oz_schur_tiles_real(mp));
  }
  return g;
}

// Algorithmic work of the fronts active at panel offset p0 (one batch member).
struct PanelWork {
  double diag_fl = 0, diag_by = 0, panel_fl = 0, panel_by = 0, schur_fl = 0, schur_by = 0;
  double off_fl = 0, off_by = 0, dpart_fl = 0, dpart_by = 0, dred_by = 0;
  double slice_off_by = 0, slice_schur_by = 0;  // split path: read FP64, write bf16 planes (10 B / element / slice)
};

// Work of the update of the rest of a panel block (columns before min(cb, s)).
void block_band_work(const Level& lv, int p0, int b, int cb, double es, double fma_fl, double& fl, double& by,
                     double& slice_by) {
  fl = by = slice_by = 0;
  for (size_t t = 0; t < lv.fronts.size(); ++t) {
    if (lv.s[t] <= p0) break;
    const double bb = std::min(b, lv.s[t] - p0), mp = double(lv.m[t]) - p0 - bb;
    const double cs = std::max(0.0, std::min(double(std::min(cb, lv.s[t])) - p0 - bb, mp));
    const double area = cs * mp - cs * (cs - 1) / 2;  // lower-triangle entries of the column band
    fl += fma_fl * area * bb;
    by += (2 * area + (mp + cs) * bb) * es;
    slice_by += (mp + cs) * bb * (es + 4.0 * 6);
  }
}

PanelWork panel_work(const Level& lv, int p0, int b, double es, double fma_fl) {
  PanelWork w;
  for (size_t t = 0; t < lv.fronts.size(); ++t) {
    if (lv.s[t] <= p0) break;
    double bb = std::min(b, lv.s[t] - p0);
    double mp = double(lv.m[t]) - p0 - bb;
    double nt = std::ceil(mp / kTile);
    w.diag_fl += fma_fl * bb * bb * bb;
    w.diag_by += 2 * bb * bb * es;
    w.panel_fl += fma_fl * mp * bb * bb;
    w.panel_by += (3 * mp * bb + bb * bb) * es;
    w.schur_fl += fma_fl * mp * (mp + 1) / 2 * bb;
    w.schur_by += (mp * (mp + 1) + 2 * mp * bb) * es;
    w.off_fl += fma_fl * mp * mp * bb;
    w.off_by += (mp * mp + 3 * mp * bb) * es;
    w.dpart_fl += fma_fl * bb * bb * mp;
    w.dpart_by += (2 * mp * bb + nt * bb * bb) * es;
    w.dred_by += (nt + 2) * bb * bb * es;
    w.slice_off_by += mp * mp * es + mp * bb * (es + 4.0 * 6);  // A: exponents only; B: slices
    w.slice_schur_by += 2 * mp * bb * (es + 4.0 * 6);
  }
  return w;
}

Profiler g_off;  // a profiler that is never switched on

// Split-precision scratch of a workspace: the complex layout (poles) or the
// real one (inertia shifts, twice as many batch members).
OzScratch split_scratch(const pexsi_plan* p, Workspace& ws, bool real) {
  return OzScratch{ws.ozA, real ? p->d_ozA_off_r : p->d_ozA_off, real ? p->ozA_stride_r : p->ozA_stride,
                   ws.ozB, real ? p->d_ozB_off_r : p->d_ozB_off, real ? p->ozB_stride_r : p->ozB_stride,
                   ws.exA, p->d_exA_off, p->exA_stride, ws.exB, p->d_exB_off, p->exB_stride,
                   ws.ozfail + (real ? 1 : 0), ws.ymax, p->d_ymax_off, p->ymax_stride, p->wait_ns,
                   p->opts.inject == 1 ? 1 : 0};
}

// Factor the batch in F (assembled), leaves to root.
template <typename T>
void factor_batch(const pexsi_plan* p, Workspace& ws, T* F, const BatchShifts& sh, bool count, Profiler& pf) {
  NvtxRange range("pexsi: multifrontal LDL^T");
  cudaStream_t st = ws.stream;
  DevFronts fr = p->fronts();
  // the inertia shifts (count) keep their own status words; their panel blocks
  // are saved and counted after the factorisation
  DevStatus status{ws.brk + (count ? 1 : 0), ws.minpiv + (count ? 1 : 0), ws.neg, count ? ws.dsave : nullptr,
                   p->d_col0, p->sym.n * int64_t(p->b)};
  const int b = p->b;
  const double es = double(sizeof(T)), fl = sizeof(T) == 16 ? 8.0 : 2.0, nb = sh.nb;
  for (size_t L = 0; L < p->levels.size(); ++L) {
    const Level& lv = p->levels[L];
    const int32_t* dfr = p->d_level_fronts + lv.front_off;
    for (size_t k = 0; k < lv.ea_off.size(); ++k) {
      cudaEvent_t a = pf.begin(st);
      launch_extend_add<T>(F, fr, p->d_ea + lv.ea_off[k], lv.ea_count[k], p->d_tile_pref + lv.ea_pref_off[k],
                           lv.ea_total[k], sh, st);
      pf.end(a, P_EXTEND, st, 0.0, nb * lv.ea_elems[k] * es);
    }
    for (int p0 = 0; p0 < lv.max_s; p0 += b) {
      PanelGeom g = panel_geom(lv, p0, b);
      PanelWork w = pf.on ? panel_work(lv, p0, b, es, fl) : PanelWork();
      cudaEvent_t a = pf.begin(st);
      launch_diag_inv<T>(F, fr, dfr, g.nact, p0, b, sh, status, count, st);
      pf.end(a, P_DIAG, st, nb * w.diag_fl, nb * w.diag_by);
      a = pf.begin(st);
      const int S = p->oz_slices;
      // executed tensor flops per algorithmic flop: S(S+1)/2 slice pairs, 4 real
      // products per complex multiply-add (8 flops) or 1 per real one (2 flops)
      const double tens = S * (S + 1) / 2.0;
      if (S > 0 && sizeof(T) == sizeof(double2)) {
        OzScratch oz = split_scratch(p, ws, false);
        launch_oz_panel(reinterpret_cast<double2*>(F), fr, dfr, g.nact, g.max_mp, p0, b, S, oz, sh.nb, st, false);
        pf.end(a, P_SLICE, st, 0.0, nb * w.slice_schur_by / 2);
        a = pf.begin(st);
        launch_oz_panel(reinterpret_cast<double2*>(F), fr, dfr, g.nact, g.max_mp, p0, b, S, oz, sh.nb, st, true);
        pf.end(a, P_PANEL, st, nb * w.panel_fl, nb * w.panel_by, 1, nb * w.panel_fl * tens);
      } else if (S > 0) {
        OzScratch oz = split_scratch(p, ws, true);
        launch_oz_panel_real(reinterpret_cast<double*>(F), fr, dfr, g.nact, g.max_mp, p0, b, S, oz, sh.nb, st, false);
        pf.end(a, P_SLICE, st, 0.0, nb * w.slice_schur_by / 2);
        a = pf.begin(st);
        launch_oz_panel_real(reinterpret_cast<double*>(F), fr, dfr, g.nact, g.max_mp, p0, b, S, oz, sh.nb, st, true);
        pf.end(a, P_PANEL, st, nb * w.panel_fl, nb * w.panel_by, 1, nb * w.panel_fl * tens);
      } else {
        launch_panel_solve<T>(F, fr, dfr, g.nact, g.row_tiles, p0, b, sh, st);
        pf.end(a, P_PANEL, st, nb * w.panel_fl, nb * w.panel_by);
      }
      if (S > 0) {
        // Blocks of p->oz_block (<= kOzBlockPanels) panels: each panel updates the rest of its
        // block (columns before min(cb, s)); after the block's last panel one
        // update with K = the block width covers everything to its right, so
        // that part of the front is read and written once per block instead
        // of once per panel.
        const bool cplx = sizeof(T) == sizeof(double2);
        const int bw = p->oz_block * b, blk0 = p0 / bw * bw, cb = blk0 + bw;
        const PanelGeom gb = panel_geom(lv, p0, b, cb);
        double band_fl, band_by, band_slice_by;
        block_band_work(lv, p0, b, cb, es, fl, band_fl, band_by, band_slice_by);
        OzScratch oz = split_scratch(p, ws, !cplx);
        if ((cplx ? gb.oz_blk : gb.oz_blk_r) > 0) {  // none at the block's last panel
          a = pf.begin(st);
          if (cplx)
            launch_oz_slice_schur(reinterpret_cast<double2*>(F), fr, dfr, g.nact, g.max_mp, p0, b, S, oz, sh.nb, st, cb);
          else
            launch_oz_slice_schur_real(reinterpret_cast<double*>(F), fr, dfr, g.nact, g.max_mp, p0, b, S, oz, sh.nb, st,
                                       cb);
          pf.end(a, P_SLICE, st, 0.0, nb * band_slice_by);
          a = pf.begin(st);
          if (cplx)
            launch_oz_gemm_schur(reinterpret_cast<double2*>(F), fr, dfr, g.nact, gb.oz_blk, p0, b, S, oz, sh.nb, st, cb);
          else
            launch_oz_gemm_schur_real(reinterpret_cast<double*>(F), fr, dfr, g.nact, gb.oz_blk_r, p0, b, S, oz, sh.nb,
                                      st, cb);
          // executed tensor flops: S(S+1)/2 slice pairs; a complex multiply-add
          // is 4 real products (8 flops counted), a real one 1 (2 flops)
          pf.end(a, P_SCHUR, st, nb * band_fl, nb * band_by, 1, nb * band_fl * tens);
        }
        if (p0 + b >= std::min(cb, lv.max_s)) {  // the level's last panel of the block
          const PanelGeom gt = panel_geom(lv, blk0, bw);
          const PanelWork wt = pf.on ? panel_work(lv, blk0, bw, es, fl) : PanelWork();
          a = pf.begin(st);
          if (cplx)
            launch_oz_slice_schur(reinterpret_cast<double2*>(F), fr, dfr, gt.nact, gt.max_mp, blk0, bw, S, oz, sh.nb, st,
                                  0);
          else
            launch_oz_slice_schur_real(reinterpret_cast<double*>(F), fr, dfr, gt.nact, gt.max_mp, blk0, bw, S, oz, sh.nb,
                                       st, 0);
          pf.end(a, P_SLICE, st, 0.0, nb * wt.slice_schur_by);
          a = pf.begin(st);
          if (cplx)
            launch_oz_gemm_schur(reinterpret_cast<double2*>(F), fr, dfr, gt.nact, gt.oz_schur, blk0, bw, S, oz, sh.nb, st,
                                 0);
          else
            launch_oz_gemm_schur_real(reinterpret_cast<double*>(F), fr, dfr, gt.nact, gt.oz_schur_r, blk0, bw, S, oz,
                                      sh.nb, st, 0);
          pf.end(a, P_SCHUR, st, nb * wt.schur_fl, nb * wt.schur_by, 1, nb * wt.schur_fl * tens);
        }
      } else {
        a = pf.begin(st);
        launch_trailing<T>(F, fr, dfr, g.nact, g.tri_tiles, p0, b, sh, st);
        pf.end(a, P_SCHUR, st, nb * w.schur_fl, nb * w.schur_by);
      }
    }
  }
  if (count) {
    cudaEvent_t a = pf.begin(st);
    launch_bk_count_all<T>(p->d_bk_slots, p->n_bk_slots, fr, b, sh.nb, status, st);
    pf.end(a, P_DIAG, st, 0.0, 0.0);
  }
  ck(cudaGetLastError(), "factor kernels");
}

void selinv_batch(const pexsi_plan* p, Workspace& ws, const BatchShifts& sh, Profiler& pf) {
  NvtxRange range("pexsi: selected inversion");
  cudaStream_t st = ws.stream;
  DevFronts fr = p->fronts();
  const int b = p->b;
  const double es = 16.0, nb = sh.nb;
  for (int L = int(p->levels.size()) - 1; L >= 0; --L) {
    const Level& lv = p->levels[L];
    const int32_t* dfr = p->d_level_fronts + lv.front_off;
    cudaEvent_t a = pf.begin(st);
    launch_gather(ws.Y, fr, dfr, int(lv.fronts.size()), p->d_tile_pref + lv.gather_pref_off, lv.gather_total, sh, st);
    pf.end(a, P_GATHER, st, 0.0, nb * lv.gather_bytes);
    if (p->oz_slices > 0) {
      int max_m = 0;
      for (int mk : lv.m) max_m = std::max(max_m, mk);
      a = pf.begin(st);
      launch_oz_rowmax_init(ws.Y, fr, dfr, int(lv.fronts.size()), max_m, split_scratch(p, ws, false), sh.nb, st);
      pf.end(a, P_SLICE, st, 0.0, nb * lv.gather_bytes);
    }
    int last = ((lv.max_s - 1) / b) * b;
    for (int p0 = last; p0 >= 0; p0 -= b) {
      PanelGeom g = panel_geom(lv, p0, b);
      PanelWork w = pf.on ? panel_work(lv, p0, b, es, 8.0) : PanelWork();
      a = pf.begin(st);
      if (p->oz_slices > 0) {
        OzScratch oz = split_scratch(p, ws, false);
        const int S = p->oz_slices;
        launch_oz_takahashi(ws.Y, ws.F, fr, dfr, g.nact, g.max_mp, p0, b, S, oz, sh.nb, st, true);
        pf.end(a, P_SLICE, st, 0.0, nb * w.slice_off_by);
        a = pf.begin(st);
        launch_oz_takahashi(ws.Y, ws.F, fr, dfr, g.nact, g.max_mp, p0, b, S, oz, sh.nb, st, false);
        pf.end(a, P_OFFDIAG, st, nb * w.off_fl, nb * w.off_by, 1, nb * w.off_fl * 4.0 * S * (S + 1) / 2 / 8.0 * 2.0);
      } else {
        launch_selinv_offdiag(ws.Y, ws.F, fr, dfr, g.nact, g.row_tiles, g.max_mp, p0, b, sh, ws.kpart, p->d_part_off,
                              kpart_stride(p), st);
        pf.end(a, P_OFFDIAG, st, nb * w.off_fl, nb * w.off_by);
      }
      if (p->oz_slices > 0) {
        const int S = p->oz_slices;
        OzScratch oz = split_scratch(p, ws, false);
        a = pf.begin(st);
        launch_oz_dpart(ws.Y, ws.F, ws.part, p->d_part_off, p->part_stride, fr, dfr, g.nact, g.max_mp, p0, b, S, oz,
                        sh.nb, st, 0);
        pf.end(a, P_SLICE, st, 0.0, nb * w.dpart_by / 2);
        a = pf.begin(st);
        launch_oz_dpart(ws.Y, ws.F, ws.part, p->d_part_off, p->part_stride, fr, dfr, g.nact, g.max_mp, p0, b, S, oz,
                        sh.nb, st, 1);
        pf.end(a, P_DPART, st, nb * w.dpart_fl, nb * w.dpart_by, 1, nb * w.dpart_fl * S * (S + 1) / 2.0);
        a = pf.begin(st);
        launch_oz_dpart(ws.Y, ws.F, ws.part, p->d_part_off, p->part_stride, fr, dfr, g.nact, g.max_mp, p0, b, S, oz,
                        sh.nb, st, 2);
        pf.end(a, P_DRED, st, 0.0, nb * w.dred_by);
      } else {
        a = pf.begin(st);
        launch_selinv_diag_partial(ws.Y, ws.F, ws.part, p->d_part_off, p->part_stride, fr, dfr, g.nact, g.row_tiles,
                                   p0, b, sh, st);
        pf.end(a, P_DPART, st, nb * w.dpart_fl, nb * w.dpart_by);
        a = pf.begin(st);
        launch_selinv_diag_reduce(ws.Y, ws.F, ws.part, p->d_part_off, p->part_stride, fr, dfr, g.nact, p0, b, sh, st);
        pf.end(a, P_DRED, st, 0.0, nb * w.dred_by);
      }
    }
  }
  ck(cudaGetLastError(), "selinv kernels");
}

BatchShifts make_shifts(const std::vector<std::complex<double>>& z, const std::vector<std::complex<double>>* wr,
                        const std::vector<std::complex<double>>* we, const std::vector<std::complex<double>>* wf,
                        int begin, int nb, const std::vector<std::complex<double>>* wd = nullptr) {
  BatchShifts sh;
  std::memset(&sh, 0, sizeof(sh));
  sh.nb = nb;
  for (int t = 0; t < nb; ++t) {
    sh.re[t] = z[begin + t].real();
    sh.im[t] = z[begin + t].imag();
    if (wr) { sh.wr_re[t] = (*wr)[begin + t].real(); sh.wr_im[t] = (*wr)[begin + t].imag(); }
    if (we) { sh.we_re[t] = (*we)[begin + t].real(); sh.we_im[t] = (*we)[begin + t].imag(); }
    if (wf) { sh.wf_re[t] = (*wf)[begin + t].real(); sh.wf_im[t] = (*wf)[begin + t].imag(); }
    if (wd) { sh.wd_re[t] = (*wd)[begin + t].real(); sh.wd_im[t] = (*wd)[begin + t].imag(); }
  }
  return sh;
}

// A bounded wait inside the split-precision kernels ran out: the site it
// gave up at, read from the status word of the chain (0 = poles, 1 = inertia).
int split_failed(Workspace& ws, int which, std::string* err, const char* what) {
  if (!ws.ozfail) return 0;
  int f = 0;
  ck(cudaMemcpyAsync(&f, ws.ozfail + which, sizeof(int), cudaMemcpyDeviceToHost, ws.stream), "status");
  ck(cudaStreamSynchronize(ws.stream), "sync");
  if (f && err)
    *err = std::string(what) + ": a bounded device-side wait ran out (mode " + std::to_string((f >> 28) & 3) +
           ", wait " + std::to_string(((f >> 20) & 255) & 15) + ", K tile " + std::to_string(((f >> 20) & 255) >> 4) +
           ", CTA " + std::to_string((f - 1) & ((1 << 20) - 1)) + ")";
  return f;
}

// One batch of complex shifts through assembly, factorisation and selected
// inversion; the result is left in ws.Y.
// Factorisation and selected inversion of the nb assembled poles in ws.F.
// Their launches depend on nb (and on the plan, the workspace's buffers and
// the Schur block width) but not on the shifts, so they are captured once
// into a CUDA graph per (nb, block width) and replayed on ws.stream: one
// launch instead of thousands, which matters for the short launches of small
// fronts. Captured on the workspace's own capture stream (the legacy default
// stream cannot capture); with the profiler on, and for the server's
// per-request workspaces (whose buffers live for one request), the kernels
// are launched directly.
void factor_selinv(const pexsi_plan* p, Workspace& ws, const BatchShifts& sh, Profiler& pf) {
  if (pf.on || !ws.use_graphs) {
    factor_batch<double2>(p, ws, ws.F, sh, false, pf);
    selinv_batch(p, ws, sh, pf);
    return;
  }
  for (Workspace::Graph& g : ws.graphs)
    if (g.nb == sh.nb && g.block == p->oz_block) {
      ck(cudaGraphLaunch(g.exec, ws.stream), "cudaGraphLaunch");
      return;
    }
  if (!ws.capture) ck(cudaStreamCreateWithFlags(&ws.capture, cudaStreamNonBlocking), "cudaStreamCreate(capture)");
  cudaStream_t run = ws.stream;
  ws.stream = ws.capture;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(ws.capture, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    try {
      factor_batch<double2>(p, ws, ws.F, sh, false, g_off);
      selinv_batch(p, ws, sh, g_off);
    } catch (...) {
      cudaStreamEndCapture(ws.capture, &graph);
      if (graph) cudaGraphDestroy(graph);
      ws.stream = run;
      throw;
    }
    e = cudaStreamEndCapture(ws.capture, &graph);
  }
  ws.stream = run;
  Workspace::Graph g{sh.nb, p->oz_block, nullptr};
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  ck(e, "CUDA graph capture of the level schedule");
  ws.graphs.push_back(g);
  ck(cudaGraphLaunch(g.exec, ws.stream), "cudaGraphLaunch");
}

void run_complex_batch(const pexsi_plan* p, Workspace& ws, const double* dH, const double* dS, const BatchShifts& sh,
                       Profiler& pf) {
  const int64_t pool = p->sym.front_elems;
  ck(cudaMemsetAsync(ws.F, 0, sizeof(double2) * size_t(pool) * sh.nb, ws.stream), "memset(F)");
  cudaEvent_t a = pf.begin(ws.stream);
  launch_assemble<double2>(ws.F, dH, dS, p->d_asm_src, p->d_asm_pos, p->nlow, pool, sh, ws.stream);
  pf.end(a, P_ASSEMBLE, ws.stream, 0.0, double(p->nlow) * (32.0 + 16.0 * sh.nb));
  factor_selinv(p, ws, sh, pf);
}

}  // namespace

int dm_range(const pexsi_plan* p, Workspace& ws, Profiler* prof, const double* dH, const double* dS, double mu,
             double beta, int P, double delta_e, int begin, int end, int accumulate, double* d_dm, double* d_edm,
             double* d_fdm, pexsi_dm_info* info, std::string* err) {
  NvtxRange range("pexsi: poles (assemble, LDL^T, selected inversion, pole sum)");
  Profiler& pf = prof ? *prof : g_off;
  std::vector<std::complex<double>> z, wr, we, wf, wd;
  int rc = pole_table(beta, delta_e, P, mu, z, wr, we, wf, &wd);
  if (rc) { *err = "bad pole-expansion parameters"; return rc; }
  const double* S = dS ? dS : p->d_ident;
  cudaStream_t st = ws.stream;
  double* d_ddm = ws.out + 3 * p->sym.nnz;
  if (info) ck(cudaEventRecord(ws.ev0, st), "event");
  // A call with accumulate = 0 starts a chain: its status words are cleared.
  // Calls that accumulate keep them, so that the call which finally reads
  // them (info != NULL) reports a breakdown or a timed-out wait of any batch
  // of the chain.
  if (!accumulate) reset_status(ws, 0);
  bool first = true;
  for (int b0 = begin; b0 < end; b0 += ws.batch) {
    int nb = std::min(ws.batch, end - b0);
    BatchShifts sh = make_shifts(z, &wr, &we, &wf, b0, nb, &wd);
    run_complex_batch(p, ws, dH, S, sh, pf);
    if (first && !accumulate && p->opts.inject == 2) {
      // fault injection (testing the status path): a breakdown of front 0 in
      // the chain's first batch, recorded from the host
      static const int kFront0 = 0;
      ck(cudaMemcpyAsync(ws.brk, &kFront0, sizeof(int), cudaMemcpyHostToDevice, st), "inject");
    }
    int overwrite = (first && !accumulate) ? 1 : 0;
    cudaEvent_t a = pf.begin(st);
    launch_pole_sum(ws.Y, p->sym.front_elems, p->d_entry_pos, p->sym.nnz, sh, overwrite, d_dm, d_edm, d_fdm, d_ddm,
                    st);
    int nout = 1 + (d_dm ? 1 : 0) + (d_edm ? 1 : 0) + (d_fdm ? 1 : 0);
    pf.end(a, P_POLESUM, st, 6.0 * nout * nb * double(p->sym.nnz),
           double(p->sym.nnz) * (8.0 + 16.0 * nb + 8.0 * nout * (overwrite ? 1 : 2)));
    first = false;
  }
  ck(cudaGetLastError(), "pole sum");
  if (!info) return PEXSI_OK;
  std::memset(info, 0, sizeof(*info));
  cudaEvent_t a = pf.begin(st);
  launch_traces(d_dm, d_edm, d_fdm, d_ddm, S, p->sym.nnz, ws.partials, p->trace_blocks, ws.trace3, st);
  pf.end(a, P_TRACE, st, 8.0 * double(p->sym.nnz), 40.0 * double(p->sym.nnz), 2);
  ck(cudaEventRecord(ws.ev1, st), "event");
  double tr[4] = {0, 0, 0, 0};
  int brk = INT_MAX;
  unsigned long long mp = 0;
  ck(cudaMemcpyAsync(tr, ws.trace3, sizeof(tr), cudaMemcpyDeviceToHost, st), "trace");
  ck(cudaMemcpyAsync(&brk, ws.brk, sizeof(int), cudaMemcpyDeviceToHost, st), "status");
  ck(cudaMemcpyAsync(&mp, ws.minpiv, sizeof(mp), cudaMemcpyDeviceToHost, st), "status");
  ck(cudaStreamSynchronize(st), "sync");
  float ms = 0;
  ck(cudaEventElapsedTime(&ms, ws.ev0, ws.ev1), "event");
  info->trace_dm_s = d_dm ? tr[0] : 0.0;
  info->trace_edm_s = d_edm ? tr[1] : 0.0;
  info->trace_fdm_s = d_fdm ? tr[2] : 0.0;
  info->trace_ddm_s = tr[3];
  std::memcpy(&info->min_pivot_ratio, &mp, sizeof(double));
  info->ms_total = ms;
  info->gemm_flops = (p->flops.factor_gemm + p->flops.selinv_gemm) * (end - begin);
  info->n_poles = end - begin;
  info->breakdown_front = brk == INT_MAX ? -1 : brk;
  if (split_failed(ws, 0, err, "split-precision GEMM")) return PEXSI_ERR_TIMEOUT;
  if (brk != INT_MAX) {
    *err = "zero or tiny pivot in front " + std::to_string(brk);
    return PEXSI_ERR_BREAKDOWN;
  }
  return PEXSI_OK;
}

int inertia_range(const pexsi_plan* p, Workspace& ws, Profiler* prof, const double* dH, const double* dS,
                  const double* shifts, int n_shifts, int64_t* counts, std::string* err) {
  NvtxRange range("pexsi: inertia shifts (real LDL^T, Bunch-Kaufman count)");
  Profiler& pf = prof ? *prof : g_off;
  const double* S = dS ? dS : p->d_ident;
  cudaStream_t st = ws.stream;
  const int64_t pool = p->sym.front_elems;
  // real fronts: the complex pool holds twice as many real ones
  const int cap = std::min(kMaxBatch, 2 * ws.batch);
  double* F = reinterpret_cast<double*>(ws.F);
  std::vector<std::complex<double>> z(n_shifts);
  for (int t = 0; t < n_shifts; ++t) z[t] = {shifts[t], 0.0};
  int brk_all = INT_MAX;
  for (int b0 = 0; b0 < n_shifts; b0 += cap) {
    int nb = std::min(cap, n_shifts - b0);
    BatchShifts sh = make_shifts(z, nullptr, nullptr, nullptr, b0, nb);
    reset_status(ws, 1);
    ck(cudaMemsetAsync(ws.neg, 0, sizeof(int) * kMaxBatch, st), "status");
    ck(cudaMemsetAsync(F, 0, sizeof(double) * size_t(pool) * nb, st), "memset(F)");
    cudaEvent_t a = pf.begin(st);
    launch_assemble<double>(F, dH, S, p->d_asm_src, p->d_asm_pos, p->nlow, pool, sh, st);
    pf.end(a, P_ASSEMBLE, st, 0.0, double(p->nlow) * (32.0 + 8.0 * nb));
    factor_batch<double>(p, ws, F, sh, true, pf);
    int neg[kMaxBatch];
    int brk = INT_MAX;
    ck(cudaMemcpyAsync(neg, ws.neg, sizeof(int) * nb, cudaMemcpyDeviceToHost, st), "D2H(counts)");
    ck(cudaMemcpyAsync(&brk, ws.brk + 1, sizeof(int), cudaMemcpyDeviceToHost, st), "status");
    ck(cudaStreamSynchronize(st), "sync");
    for (int t = 0; t < nb; ++t) counts[b0 + t] = neg[t];
    brk_all = std::min(brk_all, brk);
    if (split_failed(ws, 1, err, "split-precision GEMM (inertia)")) return PEXSI_ERR_TIMEOUT;
  }
  if (brk_all != INT_MAX) {
    *err = "zero or tiny pivot in front " + std::to_string(brk_all);
    return PEXSI_ERR_BREAKDOWN;
  }
  return PEXSI_OK;
}

int selinv_one(const pexsi_plan* p, Workspace& ws, const double* dH, const double* dS, double z_re, double z_im,
               double2* d_ainv, std::string* err) {
  std::vector<std::complex<double>> z{{z_re, z_im}};
  BatchShifts sh = make_shifts(z, nullptr, nullptr, nullptr, 0, 1);
  reset_status(ws, 0);
  run_complex_batch(p, ws, dH, dS ? dS : p->d_ident, sh, g_off);
  launch_extract(ws.Y, p->d_entry_pos, p->sym.nnz, d_ainv, ws.stream);
  ck(cudaGetLastError(), "extract");
  int brk = INT_MAX;
  ck(cudaMemcpyAsync(&brk, ws.brk, sizeof(int), cudaMemcpyDeviceToHost, ws.stream), "status");
  ck(cudaStreamSynchronize(ws.stream), "sync");
  if (split_failed(ws, 0, err, "split-precision GEMM")) return PEXSI_ERR_TIMEOUT;
  if (brk != INT_MAX) {
    *err = "zero or tiny pivot in front " + std::to_string(brk);
    return PEXSI_ERR_BREAKDOWN;
  }
  return PEXSI_OK;
}

// ------------------------------------------------------------------ LDU fronts
// Complex Hermitian H and S (Sec. IV: k-points, spin-orbit coupling). For
// Im z > 0, A = H - z S is neither Hermitian nor complex symmetric, but
// Im x^H A x = -Im z x^H S x < 0 for x != 0, so every leading block and
// Schur complement is nonsingular and A = L D U (L, U unit triangular per
// panel, D the panels' diagonal blocks) exists without pivoting across
// panels. A^{-1} = U^{-1} D^{-1} L^{-1} gives, per panel P with trailing rows S,
//   Y[S,P] = -Y[S,S] L[S,P],  Y[P,S] = -U[P,S] Y[S,S],  Y[P,P] = D^{-1} - U[P,S] Y[S,P],
// which for U = L^T is the recursion of the complex-symmetric fronts.
namespace {

void factor_batch_gen(const pexsi_plan* p, Workspace& ws, const BatchShifts& sh, bool count, Profiler& pf) {
  NvtxRange range("pexsi: multifrontal LDU");
  cudaStream_t st = ws.stream;
  DevFronts fr = p->fronts();
  DevStatus status{ws.brk + (count ? 1 : 0), ws.minpiv + (count ? 1 : 0), ws.neg, count ? ws.dsave : nullptr,
                   p->d_col0, p->sym.n * int64_t(p->b)};
  const int b = p->b;
  const double nb = sh.nb;
  for (size_t L = 0; L < p->levels.size(); ++L) {
    const Level& lv = p->levels[L];
    const int32_t* dfr = p->d_level_fronts + lv.front_off;
    for (size_t k = 0; k < lv.ea_off.size(); ++k) {
      cudaEvent_t a = pf.begin(st);
      launch_extend_add_full(ws.F, fr, p->d_ea + lv.ea_off[k], lv.ea_count[k], p->d_tile_pref + lv.ea_pref_off_full[k],
                             lv.ea_total_full[k], sh, st);
      pf.end(a, P_EXTEND, st, 0.0, nb * lv.ea_elems_full[k] * 16.0);
    }
    for (int p0 = 0; p0 < lv.max_s; p0 += b) {
      PanelGeom g = panel_geom(lv, p0, b);
      PanelWork w = pf.on ? panel_work(lv, p0, b, 16.0, 8.0) : PanelWork();
      cudaEvent_t a = pf.begin(st);
      launch_diag_inv_gen(ws.F, fr, dfr, g.nact, p0, b, sh, status, count, st);
      pf.end(a, P_DIAG, st, nb * w.diag_fl, nb * w.diag_by);
      a = pf.begin(st);
      launch_panel_solve_gen(ws.F, fr, dfr, g.nact, g.row_tiles, p0, b, sh, st, false);
      pf.end(a, P_PANEL, st, nb * w.panel_fl, nb * w.panel_by);
      a = pf.begin(st);
      launch_trailing_full(ws.F, fr, dfr, g.nact, g.row_tiles, p0, b, sh, st);
      pf.end(a, P_SCHUR, st, 2.0 * nb * w.schur_fl, 2.0 * nb * w.schur_by);
      a = pf.begin(st);
      launch_panel_solve_gen(ws.F, fr, dfr, g.nact, g.row_tiles, p0, b, sh, st, true);
      pf.end(a, P_PANEL, st, nb * w.panel_fl, nb * w.panel_by);
    }
  }
  if (count) launch_bk_count_all<double2>(p->d_bk_slots, p->n_bk_slots, fr, b, sh.nb, status, st);
  ck(cudaGetLastError(), "LDU factor kernels");
}

void selinv_batch_gen(const pexsi_plan* p, Workspace& ws, const BatchShifts& sh, Profiler& pf) {
  NvtxRange range("pexsi: two-sided selected inversion");
  cudaStream_t st = ws.stream;
  DevFronts fr = p->fronts();
  const int b = p->b;
  const double nb = sh.nb;
  for (int L = int(p->levels.size()) - 1; L >= 0; --L) {
    const Level& lv = p->levels[L];
    const int32_t* dfr = p->d_level_fronts + lv.front_off;
    cudaEvent_t a = pf.begin(st);
    launch_gather(ws.Y, fr, dfr, int(lv.fronts.size()), p->d_tile_pref + lv.gather_pref_off, lv.gather_total, sh, st);
    pf.end(a, P_GATHER, st, 0.0, nb * lv.gather_bytes);
    const int last = ((lv.max_s - 1) / b) * b;
    for (int p0 = last; p0 >= 0; p0 -= b) {
      PanelGeom g = panel_geom(lv, p0, b);
      PanelWork w = pf.on ? panel_work(lv, p0, b, 16.0, 8.0) : PanelWork();
      a = pf.begin(st);
      launch_selinv_offdiag_gen(ws.Y, ws.F, fr, dfr, g.nact, g.row_tiles, p0, b, sh, st);
      pf.end(a, P_OFFDIAG, st, 2.0 * nb * w.off_fl, 2.0 * nb * w.off_by);
      a = pf.begin(st);
      launch_selinv_diag_partial_gen(ws.Y, ws.F, ws.part, p->d_part_off, p->part_stride, fr, dfr, g.nact, g.row_tiles,
                                     p0, b, sh, st);
      pf.end(a, P_DPART, st, nb * w.dpart_fl, nb * w.dpart_by);
      a = pf.begin(st);
      launch_selinv_diag_reduce_gen(ws.Y, ws.F, ws.part, p->d_part_off, p->part_stride, fr, dfr, g.nact, p0, b, sh, st);
      pf.end(a, P_DRED, st, 0.0, nb * w.dred_by);
    }
  }
  ck(cudaGetLastError(), "LDU selinv kernels");
}

void run_gen_batch(const pexsi_plan* p, Workspace& ws, const double2* dH, const double2* dS, const BatchShifts& sh,
                   bool count, bool selinv, Profiler& pf) {
  const int64_t pool = p->sym.front_elems;
  ck(cudaMemsetAsync(ws.F, 0, sizeof(double2) * size_t(pool) * sh.nb, ws.stream), "memset(F)");
  cudaEvent_t a = pf.begin(ws.stream);
  launch_assemble_gen(ws.F, dH, dS, p->d_pos_full, p->sym.nnz, pool, sh, ws.stream);
  pf.end(a, P_ASSEMBLE, ws.stream, 0.0, double(p->sym.nnz) * (32.0 + 16.0 * sh.nb));
  factor_batch_gen(p, ws, sh, count, pf);
  if (selinv) selinv_batch_gen(p, ws, sh, pf);
}

}  // namespace

int dm_range_herm(const pexsi_plan* p, Workspace& ws, Profiler* prof, const double2* dH, const double2* dS, double mu,
                  double beta, int P, double delta_e, int begin, int end, int accumulate, double2* d_dm,
                  double2* d_edm, double2* d_fdm, pexsi_dm_info* info, std::string* err) {
  NvtxRange range("pexsi: Hermitian poles (LDU fronts)");
  Profiler& pf = prof ? *prof : g_off;
  std::vector<std::complex<double>> z, wr, we, wf, wd;
  int rc = pole_table(beta, delta_e, P, mu, z, wr, we, wf, &wd);
  if (rc) { *err = "bad pole-expansion parameters"; return rc; }
  const double2* S = dS ? dS : p->d_ident_c;
  cudaStream_t st = ws.stream;
  const int64_t nnz = p->sym.nnz;
  double2* d_ddm = p->d_hout + 3 * nnz;
  if (info) ck(cudaEventRecord(ws.ev0, st), "event");
  if (!accumulate) reset_status(ws, 0);
  bool first = true;
  for (int b0 = begin; b0 < end; b0 += ws.batch) {
    const int nb = std::min(ws.batch, end - b0);
    BatchShifts sh = make_shifts(z, &wr, &we, &wf, b0, nb, &wd);
    run_gen_batch(p, ws, dH, S, sh, false, true, pf);
    if (first && !accumulate && p->opts.inject == 2) {
      static const int kFront0 = 0;
      ck(cudaMemcpyAsync(ws.brk, &kFront0, sizeof(int), cudaMemcpyHostToDevice, st), "inject");
    }
    const int overwrite = (first && !accumulate) ? 1 : 0;
    cudaEvent_t a = pf.begin(st);
    launch_pole_sum_herm(ws.Y, p->sym.front_elems, p->d_pos_full, p->d_pos_t, nnz, sh, overwrite, d_dm, d_edm, d_fdm,
                         d_ddm, st);
    pf.end(a, P_POLESUM, st, 4.0 * 12.0 * nb * double(nnz), double(nnz) * (16.0 + 32.0 * nb + 64.0 * (overwrite ? 1 : 2)));
    first = false;
  }
  ck(cudaGetLastError(), "pole sum");
  if (!info) return PEXSI_OK;
  std::memset(info, 0, sizeof(*info));
  // Tr[X S] = sum_e X_e conj(S_e) for Hermitian S: its real part is the
  // dot product of the interleaved arrays (the imaginary part vanishes)
  cudaEvent_t a = pf.begin(st);
  launch_traces(reinterpret_cast<const double*>(d_dm), reinterpret_cast<const double*>(d_edm),
                reinterpret_cast<const double*>(d_fdm), reinterpret_cast<const double*>(d_ddm),
                reinterpret_cast<const double*>(S), 2 * nnz, ws.partials, p->trace_blocks, ws.trace3, st);
  pf.end(a, P_TRACE, st, 8.0 * double(nnz), 80.0 * double(nnz), 2);
  ck(cudaEventRecord(ws.ev1, st), "event");
  double tr[4] = {0, 0, 0, 0};
  int brk = INT_MAX;
  unsigned long long mp = 0;
  ck(cudaMemcpyAsync(tr, ws.trace3, sizeof(tr), cudaMemcpyDeviceToHost, st), "trace");
  ck(cudaMemcpyAsync(&brk, ws.brk, sizeof(int), cudaMemcpyDeviceToHost, st), "status");
  ck(cudaMemcpyAsync(&mp, ws.minpiv, sizeof(mp), cudaMemcpyDeviceToHost, st), "status");
  ck(cudaStreamSynchronize(st), "sync");
  float ms = 0;
  ck(cudaEventElapsedTime(&ms, ws.ev0, ws.ev1), "event");
  info->trace_dm_s = d_dm ? tr[0] : 0.0;
  info->trace_edm_s = d_edm ? tr[1] : 0.0;
  info->trace_fdm_s = d_fdm ? tr[2] : 0.0;
  info->trace_ddm_s = tr[3];
  std::memcpy(&info->min_pivot_ratio, &mp, sizeof(double));
  info->ms_total = ms;
  info->gemm_flops = (2.0 * p->flops.factor_gemm + 2.0 * p->flops.selinv_gemm) * (end - begin);
  info->n_poles = end - begin;
  info->breakdown_front = brk == INT_MAX ? -1 : brk;
  if (brk != INT_MAX) {
    *err = "zero or tiny pivot in front " + std::to_string(brk);
    return PEXSI_ERR_BREAKDOWN;
  }
  return PEXSI_OK;
}

// Inertia counts of the Hermitian pencil: LDU (= L D L^H) fronts of H -
// sigma S with real sigma and the Hermitian Bunch-Kaufman count of each D
// block (Sylvester's law, Haynsworth's inertia additivity, Sec. II.C).
int inertia_range_herm(const pexsi_plan* p, Workspace& ws, const double2* dH, const double2* dS, const double* shifts,
                       int n_shifts, int64_t* counts, std::string* err) {
  const double2* S = dS ? dS : p->d_ident_c;
  cudaStream_t st = ws.stream;
  std::vector<std::complex<double>> z(n_shifts);
  for (int t = 0; t < n_shifts; ++t) z[t] = {shifts[t], 0.0};
  int brk_all = INT_MAX;
  for (int b0 = 0; b0 < n_shifts; b0 += ws.batch) {
    const int nb = std::min(ws.batch, n_shifts - b0);
    BatchShifts sh = make_shifts(z, nullptr, nullptr, nullptr, b0, nb);
    reset_status(ws, 1);
    ck(cudaMemsetAsync(ws.neg, 0, sizeof(int) * kMaxBatch, st), "status");
    run_gen_batch(p, ws, dH, S, sh, true, false, g_off);
    int neg[kMaxBatch];
    int brk = INT_MAX;
    ck(cudaMemcpyAsync(neg, ws.neg, sizeof(int) * nb, cudaMemcpyDeviceToHost, st), "D2H(counts)");
    ck(cudaMemcpyAsync(&brk, ws.brk + 1, sizeof(int), cudaMemcpyDeviceToHost, st), "status");
    ck(cudaStreamSynchronize(st), "sync");
    for (int t = 0; t < nb; ++t) counts[b0 + t] = neg[t];
    brk_all = std::min(brk_all, brk);
  }
  if (brk_all != INT_MAX) {
    *err = "zero or tiny pivot in front " + std::to_string(brk_all);
    return PEXSI_ERR_BREAKDOWN;
  }
  return PEXSI_OK;
}

int selinv_one_herm(const pexsi_plan* p, Workspace& ws, const double2* dH, const double2* dS, double z_re, double z_im,
                    double2* d_ainv, std::string* err) {
  std::vector<std::complex<double>> z{{z_re, z_im}};
  BatchShifts sh = make_shifts(z, nullptr, nullptr, nullptr, 0, 1);
  reset_status(ws, 0);
  run_gen_batch(p, ws, dH, dS ? dS : p->d_ident_c, sh, false, true, g_off);
  launch_extract(ws.Y, p->d_pos_full, p->sym.nnz, d_ainv, ws.stream);
  ck(cudaGetLastError(), "extract");
  int brk = INT_MAX;
  ck(cudaMemcpyAsync(&brk, ws.brk, sizeof(int), cudaMemcpyDeviceToHost, ws.stream), "status");
  ck(cudaStreamSynchronize(ws.stream), "sync");
  if (brk != INT_MAX) {
    *err = "zero or tiny pivot in front " + std::to_string(brk);
    return PEXSI_ERR_BREAKDOWN;
  }
  return PEXSI_OK;
}

// ------------------------------------------------------------------ groups of systems
// Several systems side by side in one plan: their fronts are concatenated
// into one pool and their elimination trees into one forest, so that every
// launch of the level schedule (block inverses, panel solves, Schur
// updates, Takahashi steps) covers the fronts of all systems at that height
// of their trees, for all poles of a wave. Only assembly and the pole sum
// are per system (each system has its own values, shifts and weights). The
// poles and the systems are independent (Sec. II.B): the merged forest
// computes exactly what the systems compute alone.
Symbolic merge_symbolic(const std::vector<const Symbolic*>& parts) {
  Symbolic m;
  int64_t off_n = 0, off_rows = 0, off_pool = 0;
  int32_t off_super = 0, hmax = 0;
  for (const Symbolic* q : parts) hmax = std::max(hmax, q->nlevels);
  for (const Symbolic* q : parts) {
    for (int32_t v : q->perm) m.perm.push_back(v + int32_t(off_n));
    for (int32_t v : q->iperm) m.iperm.push_back(v + int32_t(off_n));
    for (int32_t K = 0; K < q->nsuper; ++K) {
      m.first.push_back(q->first[K] + int32_t(off_n));
      m.rptr.push_back(q->rptr[K] + off_rows);
      m.parent.push_back(q->parent[K] >= 0 ? q->parent[K] + off_super : -1);
      m.height.push_back(q->height[K] + hmax - q->nlevels);
      m.front_off.push_back(q->front_off[K] + off_pool);
    }
    for (int32_t v : q->rows) m.rows.push_back(v + int32_t(off_n));
    m.rel.insert(m.rel.end(), q->rel.begin(), q->rel.end());
    for (int64_t v : q->entry_pos) m.entry_pos.push_back(v + off_pool);
    for (int64_t v : q->entry_pos_up) m.entry_pos_up.push_back(v + off_pool);
    m.entry_lower.insert(m.entry_lower.end(), q->entry_lower.begin(), q->entry_lower.end());
    // levels aligned at the roots: system q's level L becomes L + (H - H_q)
    // (H the tallest tree), so that the widest fronts -- the roots and the
    // separators just below them, which hold most panels -- of every system
    // share launches; shifting a whole tree keeps its children before parents
    if (int32_t(m.level_fronts.size()) < hmax) m.level_fronts.resize(hmax);
    for (int32_t L = 0; L < q->nlevels; ++L)
      for (int32_t K : q->level_fronts[L]) m.level_fronts[L + hmax - q->nlevels].push_back(K + off_super);
    m.nnz += q->nnz;
    m.nnz_L += q->nnz_L;
    m.max_front = std::max(m.max_front, q->max_front);
    m.max_width = std::max(m.max_width, q->max_width);
    off_n += q->n;
    off_rows += int64_t(q->rows.size());
    off_pool += q->front_elems;
    off_super += q->nsuper;
  }
  m.n = off_n;
  m.nsuper = off_super;
  m.first.push_back(int32_t(off_n));
  m.rptr.push_back(off_rows);
  m.front_off.push_back(off_pool);
  m.front_elems = off_pool;
  m.nlevels = int32_t(m.level_fronts.size());
  return m;
}

// Poles [begin, end) of every system of a merged plan, in waves of `wave`
// poles: dH[q], dS[q] (NULL = I) the values of system q, mu[q], beta[q],
// delta_e[q] its expansion (P poles each), d_dm[q] / d_edm[q] / d_fdm[q] its
// outputs (any may be NULL). info (nsys entries, NULL = do not wait) gets
// each system's traces; status rules as dm_range.
int dm_range_group(const pexsi_plan* p, Workspace& ws, Profiler* prof, int wave, const double* const* dH,
                   const double* const* dS, const double* mu, const double* beta, int P, const double* delta_e,
                   int begin, int end, int accumulate, double* const* d_dm, double* const* d_edm, double* const* d_fdm,
                   pexsi_dm_info* info, const std::vector<int32_t>& f_off, std::string* err) {
  NvtxRange range("pexsi: group of systems (merged forest)");
  Profiler& pf = prof ? *prof : g_off;
  const int nsys = int(p->sys_entry_off.size()) - 1;
  std::vector<std::vector<std::complex<double>>> z(nsys), wr(nsys), we(nsys), wf(nsys), wd(nsys);
  for (int q = 0; q < nsys; ++q) {
    int rc = pole_table(beta[q], delta_e[q], P, mu[q], z[q], wr[q], we[q], wf[q], &wd[q]);
    if (rc) { *err = "bad pole-expansion parameters of system " + std::to_string(q); return rc; }
  }
  cudaStream_t st = ws.stream;
  const int64_t pool = p->sym.front_elems, nnz_all = p->sym.nnz;
  wave = std::max(1, std::min(wave > 0 ? wave : ws.batch, ws.batch));
  if (info) ck(cudaEventRecord(ws.ev0, st), "event");
  if (!accumulate) reset_status(ws, 0);
  bool first = true;
  for (int b0 = begin; b0 < end; b0 += wave) {
    const int nb = std::min(wave, end - b0);
    ck(cudaMemsetAsync(ws.F, 0, sizeof(double2) * size_t(pool) * nb, st), "memset(F)");
    std::vector<BatchShifts> sh(nsys);
    for (int q = 0; q < nsys; ++q) {
      sh[q] = make_shifts(z[q], &wr[q], &we[q], &wf[q], b0, nb, &wd[q]);
      const int64_t a0 = p->sys_asm_off[q], na = p->sys_asm_off[q + 1] - a0;
      const double* S = dS[q] ? dS[q] : p->d_ident + p->sys_entry_off[q];
      cudaEvent_t a = pf.begin(st);
      launch_assemble<double2>(ws.F, dH[q], S, p->d_asm_src + a0, p->d_asm_pos + a0, na, pool, sh[q], st);
      pf.end(a, P_ASSEMBLE, st, 0.0, double(na) * (32.0 + 16.0 * nb));
    }
    factor_selinv(p, ws, sh[0], pf);
    const int overwrite = (first && !accumulate) ? 1 : 0;
    for (int q = 0; q < nsys; ++q) {
      const int64_t e0 = p->sys_entry_off[q], ne = p->sys_entry_off[q + 1] - e0;
      cudaEvent_t a = pf.begin(st);
      launch_pole_sum(ws.Y, pool, p->d_entry_pos + e0, ne, sh[q], overwrite, d_dm[q], d_edm[q], d_fdm[q],
                      ws.out + 3 * nnz_all + e0, st);
      pf.end(a, P_POLESUM, st, 24.0 * nb * double(ne), double(ne) * (8.0 + 16.0 * nb + 32.0 * (overwrite ? 1 : 2)));
    }
    first = false;
  }
  ck(cudaGetLastError(), "group pole sum");
  if (!info) return PEXSI_OK;
  std::vector<double> tr(4 * size_t(nsys), 0.0);
  for (int q = 0; q < nsys; ++q) {
    const int64_t e0 = p->sys_entry_off[q], ne = p->sys_entry_off[q + 1] - e0;
    const double* S = dS[q] ? dS[q] : p->d_ident + e0;
    launch_traces(d_dm[q], d_edm[q], d_fdm[q], ws.out + 3 * nnz_all + e0, S, ne, ws.partials, p->trace_blocks,
                  ws.trace3, st);
    ck(cudaMemcpyAsync(tr.data() + 4 * q, ws.trace3, 4 * sizeof(double), cudaMemcpyDeviceToHost, st), "trace");
  }
  ck(cudaEventRecord(ws.ev1, st), "event");
  int brk = INT_MAX;
  ck(cudaMemcpyAsync(&brk, ws.brk, sizeof(int), cudaMemcpyDeviceToHost, st), "status");
  ck(cudaStreamSynchronize(st), "sync");
  float ms = 0;
  ck(cudaEventElapsedTime(&ms, ws.ev0, ws.ev1), "event");
  const int bsys = brk == INT_MAX ? -1 : int(std::upper_bound(f_off.begin(), f_off.end(), brk) - f_off.begin()) - 1;
  for (int q = 0; q < nsys; ++q) {
    pexsi_dm_info& in = info[q];
    std::memset(&in, 0, sizeof(in));
    in.trace_dm_s = d_dm[q] ? tr[4 * q] : 0.0;
    in.trace_edm_s = d_edm[q] ? tr[4 * q + 1] : 0.0;
    in.trace_fdm_s = d_fdm[q] ? tr[4 * q + 2] : 0.0;
    in.trace_ddm_s = tr[4 * q + 3];
    in.ms_total = ms;
    in.n_poles = end - begin;
    in.breakdown_front = bsys == q ? brk - f_off[q] : -1;
  }
  if (split_failed(ws, 0, err, "split-precision GEMM")) return PEXSI_ERR_TIMEOUT;
  if (brk != INT_MAX) {
    *err = "zero or tiny pivot in front " + std::to_string(brk - f_off[bsys]) + " of system " + std::to_string(bsys);
    return PEXSI_ERR_BREAKDOWN;
  }
  return PEXSI_OK;
}

}  // namespace pexsi

using namespace pexsi;

namespace {

void free_plan_device(pexsi_plan* p) {
  void* ptrs[] = {p->d_front_off, p->d_s, p->d_m, p->d_parent, p->d_rel, p->d_rptr, p->d_asm_src, p->d_asm_pos,
                  p->d_entry_pos, p->d_level_fronts, p->d_ea, p->d_tile_pref, p->d_part_off, p->d_ident,
                  p->d_ozA_off, p->d_ozB_off, p->d_exA_off, p->d_exB_off, p->d_ozA_off_r, p->d_ozB_off_r,
                  p->d_ymax_off, p->d_pos_full, p->d_pos_t, p->d_ident_c, p->d_hH, p->d_hS, p->d_hout,
                  p->d_col0, p->d_bk_slots};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  cudaStream_t st = p->ws.stream;
  workspace_free(p->ws);
  p->prof.destroy();
  if (st) cudaStreamDestroy(st);
}

int fail(pexsi_plan* p, int code, const std::string& msg) {
  if (p) p->last_error = msg;
  return code;
}

int map_cuda(pexsi_plan* p, const CudaError& ce) {
  return fail(p, PEXSI_ERR_CUDA, std::string(ce.what) + ": " + cudaGetErrorString(ce.e));
}

template <typename T>
T* dev_upload(const std::vector<T>& h) {
  T* d = nullptr;
  size_t bytes = sizeof(T) * (h.empty() ? 1 : h.size());
  ck(cudaMalloc(&d, bytes), "cudaMalloc(plan)");
  if (!h.empty()) ck(cudaMemcpy(d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice), "cudaMemcpy(plan)");
  return d;
}

void build_levels(pexsi_plan* p, std::vector<int32_t>& level_fronts, std::vector<int32_t>& ea,
                  std::vector<int64_t>& part_off,
                  std::vector<int32_t>& tile_pref) {
  const Symbolic& S = p->sym;
  const int b = p->b;
  p->levels.assign(S.nlevels, Level());
  part_off.assign(S.nsuper, 0);
  p->part_stride = 0;
  std::vector<std::vector<int32_t>> kids(S.nsuper);
  for (int32_t K = 0; K < S.nsuper; ++K)
    if (S.parent[K] >= 0) kids[S.parent[K]].push_back(K);
  for (int L = 0; L < S.nlevels; ++L) {
    Level& lv = p->levels[L];
    std::vector<int32_t> fr = S.level_fronts[L];
    std::stable_sort(fr.begin(), fr.end(), [&](int32_t a, int32_t c) { return S.s(a) > S.s(c); });
    lv.front_off = int64_t(level_fronts.size());
    lv.fronts = fr;
    lv.gather_pref_off = int64_t(tile_pref.size());
    tile_pref.push_back(0);
    int64_t slots = 0;
    for (int32_t K : fr) {
      lv.s.push_back(S.s(K));
      lv.m.push_back(S.m(K));
      lv.max_s = std::max(lv.max_s, S.s(K));
      level_fronts.push_back(K);
      int64_t r = S.r(K);
      lv.gather_tiles = std::max<int64_t>(lv.gather_tiles, ((r + 31) / 32) * ((r + 31) / 32));
      lv.gather_total += S.parent[K] >= 0 ? ((r + 31) / 32) * ((r + 31) / 32) : 0;
      tile_pref.push_back(int32_t(lv.gather_total));
      if (S.parent[K] >= 0) lv.gather_bytes += 2.0 * 16.0 * double(r) * double(r);
      int64_t first_mp = S.m(K) - std::min(b, S.s(K));
      part_off[K] = slots * int64_t(b) * b;
      slots += (first_mp + kTile - 1) / kTile;
    }
    p->part_stride = std::max<int64_t>(p->part_stride, slots * int64_t(b) * b);
    size_t maxk = 0;
    for (int32_t K : fr) maxk = std::max(maxk, kids[K].size());
    for (size_t k = 0; k < maxk; ++k) {
      lv.ea_off.push_back(int64_t(ea.size()));
      lv.ea_pref_off.push_back(int64_t(tile_pref.size()));
      tile_pref.push_back(0);
      int64_t total = 0;
      int32_t cnt = 0, tiles = 0;
      double elems = 0;
      for (int32_t K : fr) {
        if (k >= kids[K].size()) continue;
        int32_t c = kids[K][k];
        ea.push_back(c);
        ++cnt;
        int32_t r = S.r(c), T = (r + 31) / 32;
        tiles = std::max(tiles, T * (T + 1) / 2);
        total += T * (T + 1) / 2;
        tile_pref.push_back(int32_t(total));
        elems += 3.0 * double(r) * (r + 1) / 2;
      }
      lv.ea_total.push_back(total);
      lv.ea_elems.push_back(elems);
      lv.ea_count.push_back(cnt);
      lv.ea_tiles.push_back(tiles);
      // whole-square tiles of the same children (LDU fronts)
      lv.ea_pref_off_full.push_back(int64_t(tile_pref.size()));
      tile_pref.push_back(0);
      int64_t total_full = 0;
      double elems_full = 0;
      for (int32_t K : fr) {
        if (k >= kids[K].size()) continue;
        int32_t r = S.r(kids[K][k]), T = (r + 31) / 32;
        total_full += int64_t(T) * T;
        tile_pref.push_back(int32_t(total_full));
        elems_full += 3.0 * double(r) * r;
      }
      lv.ea_total_full.push_back(total_full);
      lv.ea_elems_full.push_back(elems_full);
    }
  }
  if (p->part_stride == 0) p->part_stride = int64_t(b) * b;
}

// Split-precision scratch layout: per level, the fronts' slice tiles are laid
// out one after another (only one level is active at a time).
void build_split_layout(pexsi_plan* p, std::vector<int64_t>& a_off, std::vector<int64_t>& b_off,
                        std::vector<int64_t>& ea_off, std::vector<int64_t>& eb_off, std::vector<int64_t>& ar,
                        std::vector<int64_t>& br) {
  const Symbolic& S = p->sym;
  const int b = p->b;
  ar.assign(S.nsuper, 0);
  br.assign(S.nsuper, 0);
  a_off.assign(S.nsuper, 0);
  b_off.assign(S.nsuper, 0);
  ea_off.assign(S.nsuper, 0);
  eb_off.assign(S.nsuper, 0);
  for (const Level& lv : p->levels) {
    int64_t sa = 0, sb = 0, xa = 0, xb = 0, sar = 0, sbr = 0;
    for (int32_t K : lv.fronts) {
      int64_t mp = S.m(K) - std::min(b, S.s(K));
      a_off[K] = sa;
      b_off[K] = sb;
      ea_off[K] = xa;
      eb_off[K] = xb;
      ar[K] = sar;
      br[K] = sbr;
      // the Schur update after a block of panels has K = the block width
      const int kw = std::min(kOzBlockPanels * b, S.s(K));
      sa += oz_front_bytes_A(mp, kw, p->oz_slices);
      sb += oz_front_bytes_B(mp, kw, p->oz_slices);
      sar += oz_front_bytes_A_real(mp, kw, p->oz_slices);
      sbr += oz_front_bytes_B_real(mp, kw, p->oz_slices);
      xa += std::max<int64_t>(b, mp);  // rows of A, or the panel columns (Y[S,P] exponents)
      xb += std::max<int64_t>(b, mp);
    }
    p->ozA_stride = std::max(p->ozA_stride, sa);
    p->ozB_stride = std::max(p->ozB_stride, sb);
    p->ozA_stride_r = std::max(p->ozA_stride_r, sar);
    p->ozB_stride_r = std::max(p->ozB_stride_r, sbr);
    p->exA_stride = std::max(p->exA_stride, xa);
    p->exB_stride = std::max(p->exB_stride, xb);
  }
  p->ozA_stride = std::max<int64_t>(p->ozA_stride, 16);
  p->ozB_stride = std::max<int64_t>(p->ozB_stride, 16);
  p->ozA_stride_r = std::max<int64_t>(p->ozA_stride_r, 16);
  p->ozB_stride_r = std::max<int64_t>(p->ozB_stride_r, 16);
  p->exA_stride = std::max<int64_t>(p->exA_stride, 1);
  p->exB_stride = std::max<int64_t>(p->exB_stride, 1);
}

// The plan's own workspace: the largest batch that fits the budget.
int ensure_workspace(pexsi_plan* p) {
  if (p->ws.batch > 0) return PEXSI_OK;
  size_t free_b = 0, total_b = 0;
  ck(cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo");
  int64_t budget = p->opts.hbm_budget > 0 ? p->opts.hbm_budget : int64_t(0.6 * double(free_b));
  int64_t nb = (budget - bytes_fixed(p)) / std::max<int64_t>(bytes_per_pole(p), 1);
  if (p->opts.max_batch > 0) nb = std::min<int64_t>(nb, p->opts.max_batch);
  nb = std::min<int64_t>(nb, kMaxBatch);
  if (nb < 1) return fail(p, PEXSI_ERR_NOMEM, "device workspace for one pole exceeds the HBM budget");
  workspace_alloc(p, p->ws, int(nb), p->ws.stream, false);
  return PEXSI_OK;
}

// Options of a new plan: defaults for zero fields, then validation.
int init_opts(pexsi_plan* p, const pexsi_opts* opts) {
  pexsi_opts_default(&p->opts);
  if (opts) {
    p->opts = *opts;
    pexsi_opts def;
    pexsi_opts_default(&def);
    if (p->opts.panel <= 0) p->opts.panel = def.panel;
    if (p->opts.leaf_cols <= 0) p->opts.leaf_cols = def.leaf_cols;
  }
  // the split-precision path tiles the panel as one 64-wide block
  if (p->opts.panel < 16 || p->opts.panel > 64 || p->opts.split_slices < 0 || p->opts.split_slices > 6 ||
      p->opts.split_slices == 1 || (p->opts.split_slices > 0 && p->opts.panel != 64))
    return PEXSI_ERR_INVALID_ARG;
  if (p->opts.wait_ns < 0 || p->opts.inject < 0 || p->opts.inject > 2 || p->opts.split_block < 0 ||
      p->opts.split_block > kOzBlockPanels)
    return PEXSI_ERR_INVALID_ARG;
  p->oz_block = p->opts.split_block > 0 ? p->opts.split_block : kOzBlockPanels;
  p->wait_ns = p->opts.wait_ns > 0 ? uint64_t(p->opts.wait_ns) : 1000000000ull;
  p->oz_slices = p->opts.split_slices;
  p->b = p->opts.panel;
  return PEXSI_OK;
}

// Device part of a plan whose symbolic structure, options and diagonal
// entries are set: level schedule, front maps, split-precision layout, the
// identity overlap and the plan's stream.
int upload_plan(pexsi_plan* p) {
  ck(cudaSetDevice(p->opts.device), "cudaSetDevice");
  ck(configure_kernels(p->b), "cudaFuncSetAttribute");
  if (p->oz_slices > 0) ck(oz_configure(p->oz_slices), "cudaFuncSetAttribute(split)");
  const Symbolic& S = p->sym;
  std::vector<int32_t> hs(S.nsuper), hm(S.nsuper);
  for (int32_t K = 0; K < S.nsuper; ++K) { hs[K] = S.s(K); hm[K] = S.m(K); }
  std::vector<int32_t> level_fronts, ea, tile_pref;
  std::vector<int64_t> part_off;
  build_levels(p, level_fronts, ea, part_off, tile_pref);
  for (const Level& lv : p->levels)
    if (lv.fronts.size() > 65535) {  // grid.y limit of the per-level launches
      return PEXSI_ERR_INTERNAL;
    }
  // assembly list: the lower-triangle copy of each entry; a plan that merges
  // several systems indexes each system's own value arrays, so the source
  // index is local to its system, and each system's range of the list is kept
  std::vector<int64_t> asm_src, asm_pos;
  if (p->sys_entry_off.empty()) p->sys_entry_off = {0, S.nnz};
  const size_t nsys = p->sys_entry_off.size() - 1;
  p->sys_asm_off.assign(nsys + 1, 0);
  for (size_t q = 0; q < nsys; ++q) {
    p->sys_asm_off[q] = int64_t(asm_src.size());
    for (int64_t e = p->sys_entry_off[q]; e < p->sys_entry_off[q + 1]; ++e)
      if (S.entry_lower[e]) {
        asm_src.push_back(e - p->sys_entry_off[q]);
        asm_pos.push_back(S.entry_pos[e]);
      }
  }
  p->sys_asm_off[nsys] = int64_t(asm_src.size());
  p->nlow = int64_t(asm_src.size());
  p->d_front_off = dev_upload(S.front_off);
  p->d_s = dev_upload(hs);
  p->d_m = dev_upload(hm);
  p->d_parent = dev_upload(S.parent);
  p->d_rptr = dev_upload(S.rptr);
  p->d_rel = dev_upload(S.rel);
  p->d_asm_src = dev_upload(asm_src);
  p->d_asm_pos = dev_upload(asm_pos);
  p->d_entry_pos = dev_upload(S.entry_pos);
  p->d_level_fronts = dev_upload(level_fronts);
  p->d_ea = dev_upload(ea);
  p->d_tile_pref = dev_upload(tile_pref);
  p->d_part_off = dev_upload(part_off);
  {
    std::vector<int32_t> col0(S.nsuper), slots;
    for (int32_t K = 0; K < S.nsuper; ++K) {
      col0[K] = S.first[K];
      for (int32_t p0 = 0; p0 < S.s(K); p0 += p->b) {
        slots.push_back(K);
        slots.push_back(p0);
      }
    }
    p->d_col0 = dev_upload(col0);
    p->d_bk_slots = dev_upload(slots);
    p->n_bk_slots = int32_t(slots.size() / 2);
  }
  if (p->oz_slices > 0) {
    std::vector<int64_t> oa, ob, xa, xb, ra, rb;
    build_split_layout(p, oa, ob, xa, xb, ra, rb);
    p->d_ozA_off = dev_upload(oa);
    p->d_ozB_off = dev_upload(ob);
    p->d_ozA_off_r = dev_upload(ra);
    p->d_ozB_off_r = dev_upload(rb);
    p->d_exA_off = dev_upload(xa);
    p->d_exB_off = dev_upload(xb);
    std::vector<int64_t> yo(S.nsuper);
    for (int64_t K = 0; K < S.nsuper; ++K) {
      yo[K] = p->ymax_stride;
      p->ymax_stride += S.m(K);
    }
    p->d_ymax_off = dev_upload(yo);
  }
  {
    std::vector<double> ident(S.nnz, 0.0);  // S = I on the pattern
    for (int64_t e : p->diag_entries) ident[e] = 1.0;
    p->d_ident = dev_upload(ident);
  }
  ck(cudaStreamCreateWithFlags(&p->ws.stream, cudaStreamNonBlocking), "cudaStreamCreate");
  return PEXSI_OK;
}

}  // namespace

int pexsi::plan_workspace(pexsi_plan* p) { return ensure_workspace(p); }

// Maps and staging of the Hermitian variant, made on its first call: the
// front position of every CSC entry (its own triangle) and of its transpose,
// a complex identity for S = I, and complex staging for the host calls.
int pexsi::hermitian_prepare(pexsi_plan* p) {
  if (p->d_pos_full) return PEXSI_OK;
  const Symbolic& S = p->sym;
  const size_t nnz = size_t(S.nnz);
  std::vector<int64_t> full(nnz), tr(nnz);
  for (size_t e = 0; e < nnz; ++e) {
    full[e] = S.entry_lower[e] ? S.entry_pos[e] : S.entry_pos_up[e];
    tr[e] = S.entry_lower[e] ? S.entry_pos_up[e] : S.entry_pos[e];
  }
  std::vector<double2> ident(nnz, make_double2(0.0, 0.0));
  for (int64_t e : p->diag_entries) ident[e].x = 1.0;
  p->d_pos_full = dev_upload(full);
  p->d_pos_t = dev_upload(tr);
  p->d_ident_c = dev_upload(ident);
  ck(cudaMalloc(&p->d_hH, sizeof(double2) * nnz), "cudaMalloc(hermitian staging)");
  ck(cudaMalloc(&p->d_hS, sizeof(double2) * nnz), "cudaMalloc(hermitian staging)");
  ck(cudaMalloc(&p->d_hout, sizeof(double2) * nnz * 4), "cudaMalloc(hermitian staging)");
  return PEXSI_OK;
}

namespace {

// Runs fn with the plan's workspace temporarily on `stream`: the caller's
// stream of a device-buffer call, NULL being the legacy default stream (as
// the header states), so that the caller's events on that stream bracket
// the work. The plan's own stream serves the host-buffer calls.
template <typename Fn>
int on_stream(pexsi_plan* p, void* stream, Fn fn) {
  cudaStream_t own = p->ws.stream;
  p->ws.stream = static_cast<cudaStream_t>(stream);
  int rc;
  try {
    rc = fn();
  } catch (...) {
    p->ws.stream = own;
    throw;
  }
  p->ws.stream = own;
  return rc;
}

}  // namespace

extern "C" {

int pexsi_opts_default(pexsi_opts* o) {
  if (!o) return PEXSI_ERR_INVALID_ARG;
  std::memset(o, 0, sizeof(*o));
  o->device = 0;
  o->panel = 64;
  o->leaf_cols = 96;
  o->amalgamate = 1;
  return PEXSI_OK;
}

int pexsi_profile_enable(pexsi_plan* p, int32_t on) {
  if (!p) return PEXSI_ERR_INVALID_ARG;
  try {
    if (!on) p->prof.drain();
  } catch (const CudaError& ce) {
    return map_cuda(p, ce);
  }
  p->prof.on = on != 0 && p->opts.device >= 0;
  return PEXSI_OK;
}

int pexsi_profile_reset(pexsi_plan* p) {
  if (!p) return PEXSI_ERR_INVALID_ARG;
  try {
    p->prof.reset();
  } catch (const CudaError& ce) {
    return map_cuda(p, ce);
  }
  return PEXSI_OK;
}

int pexsi_profile_read(pexsi_plan* p, pexsi_kernel_profile* out) {
  if (!p || !out) return PEXSI_ERR_INVALID_ARG;
  try {
    p->prof.drain();
  } catch (const CudaError& ce) {
    return map_cuda(p, ce);
  }
  for (int c = 0; c < PEXSI_PROFILE_CLASSES; ++c) {
    std::memset(&out[c], 0, sizeof(out[c]));
    std::strncpy(out[c].name, kProfNames[c], sizeof(out[c].name) - 1);
    out[c].launches = p->prof.launches[c];
    out[c].ms = p->prof.ms[c];
    out[c].flops = p->prof.flops[c];
    out[c].bytes = p->prof.bytes[c];
    out[c].tensor_flops = p->prof.tensor[c];
  }
  return PEXSI_OK;
}

const char* pexsi_strerror(int code) {
  switch (code) {
    case PEXSI_OK: return "ok";
    case PEXSI_ERR_INVALID_ARG: return "invalid argument";
    case PEXSI_ERR_NOT_SYMMETRIC: return "pattern not structurally symmetric";
    case PEXSI_ERR_NOMEM: return "out of memory";
    case PEXSI_ERR_CUDA: return "CUDA error";
    case PEXSI_ERR_BREAKDOWN: return "factorisation breakdown (zero or tiny pivot)";
    case PEXSI_ERR_INTERNAL: return "internal error";
    case PEXSI_ERR_CANCELLED: return "request cancelled";
    case PEXSI_ERR_TIMEOUT: return "a bounded device-side wait ran out";
    case PEXSI_PENDING: return "request pending";
    default: return "unknown error";
  }
}

const char* pexsi_last_error_detail(const pexsi_plan* p) { return p ? p->last_error.c_str() : ""; }

int pexsi_pole_table(double beta, double delta_e, int32_t n_poles, double mu, double* z, double* w_rho, double* w_E,
                     double* w_F) {
  if (!z) return PEXSI_ERR_INVALID_ARG;
  std::vector<std::complex<double>> zz, wr, we, wf;
  int rc = pole_table(beta, delta_e, n_poles, mu, zz, wr, we, wf);
  if (rc) return rc;
  for (int l = 0; l < n_poles; ++l) {
    z[2 * l] = zz[l].real(); z[2 * l + 1] = zz[l].imag();
    if (w_rho) { w_rho[2 * l] = wr[l].real(); w_rho[2 * l + 1] = wr[l].imag(); }
    if (w_E) { w_E[2 * l] = we[l].real(); w_E[2 * l + 1] = we[l].imag(); }
    if (w_F) { w_F[2 * l] = wf[l].real(); w_F[2 * l + 1] = wf[l].imag(); }
  }
  return PEXSI_OK;
}

int pexsi_setup(int64_t n, const int64_t* colptr, const int32_t* rowind, const int32_t* perm_or_null,
                const pexsi_opts* opts, pexsi_plan** out) {
  if (!out) return PEXSI_ERR_INVALID_ARG;
  *out = nullptr;
  pexsi_plan* p = nullptr;
  try {
    p = new pexsi_plan();
    int rc = init_opts(p, opts);
    if (rc) {
      delete p;
      return rc;
    }
    std::string err;
    {
      NvtxRange range("pexsi: ordering and symbolic analysis");
      rc = analyse(n, colptr, rowind, perm_or_null, p->opts.leaf_cols, p->opts.amalgamate != 0, p->sym, err);
    }
    if (rc) {
      delete p;
      return rc;
    }
    p->flops = count_flops(p->sym, p->b);
    for (int64_t j = 0; j < n; ++j)
      for (int64_t e = colptr[j]; e < colptr[j + 1]; ++e)
        if (rowind[e] == j) p->diag_entries.push_back(e);
    if (p->opts.device < 0) {  // host-only plan: symbolic analysis only
      *out = p;
      return PEXSI_OK;
    }
    rc = upload_plan(p);
    if (rc) {
      free_plan_device(p);
      delete p;
      return rc;
    }
    *out = p;
    return PEXSI_OK;
  } catch (const CudaError&) {
    if (p) { free_plan_device(p); delete p; }
    return PEXSI_ERR_CUDA;
  } catch (const std::bad_alloc&) {
    if (p) { free_plan_device(p); delete p; }
    return PEXSI_ERR_NOMEM;
  }
}

int pexsi_plan_destroy(pexsi_plan* p) {
  if (!p) return PEXSI_OK;
  if (p->opts.device >= 0) {
    cudaSetDevice(p->opts.device);
    free_plan_device(p);
  }
  delete p;
  return PEXSI_OK;
}

int pexsi_plan_get_stats(const pexsi_plan* p, pexsi_plan_stats* st) {
  if (!p || !st) return PEXSI_ERR_INVALID_ARG;
  const Symbolic& S = p->sym;
  st->n = S.n;
  st->nnz = S.nnz;
  st->nsuper = S.nsuper;
  st->nlevels = S.nlevels;
  st->nnz_L = S.nnz_L;
  st->front_elems = S.front_elems;
  st->max_front = S.max_front;
  st->max_width = S.max_width;
  st->factor_gemm_flops = p->flops.factor_gemm;
  st->selinv_gemm_flops = p->flops.selinv_gemm;
  st->diag_flops = p->flops.diag;
  st->gather_bytes = p->flops.gather_bytes;
  st->batch = p->ws.batch;
  st->workspace_bytes = p->ws.bytes;
  return PEXSI_OK;
}

int pexsi_plan_get_supernodes(const pexsi_plan* p, int32_t* first, int64_t* rptr, int32_t* rows, int32_t* parent) {
  if (!p || !first || !rptr || !parent) return PEXSI_ERR_INVALID_ARG;
  const Symbolic& S = p->sym;
  std::memcpy(first, S.first.data(), sizeof(int32_t) * (S.nsuper + 1));
  std::memcpy(rptr, S.rptr.data(), sizeof(int64_t) * (S.nsuper + 1));
  std::memcpy(parent, S.parent.data(), sizeof(int32_t) * S.nsuper);
  if (rows) std::memcpy(rows, S.rows.data(), sizeof(int32_t) * S.rows.size());
  return PEXSI_OK;
}

int pexsi_plan_get_perm(const pexsi_plan* p, int32_t* perm) {
  if (!p || !perm) return PEXSI_ERR_INVALID_ARG;
  std::memcpy(perm, p->sym.perm.data(), sizeof(int32_t) * p->sym.n);
  return PEXSI_OK;
}

int pexsi_dm_device(pexsi_plan* p, const double* dH, const double* dS, double mu, double beta, int32_t n_poles,
                    double delta_e, int32_t pole_begin, int32_t pole_end, int32_t accumulate, double* d_dm,
                    double* d_edm, double* d_fdm, void* stream, pexsi_dm_info* info) {
  if (p && p->opts.device < 0) return fail(p, PEXSI_ERR_INVALID_ARG, "host-only plan has no device");
  if (!p || !dH) return fail(p, PEXSI_ERR_INVALID_ARG, "NULL plan or H");
  if (pole_begin < 0 || pole_end > n_poles || pole_begin >= pole_end)
    return fail(p, PEXSI_ERR_INVALID_ARG, "bad pole range");
  try {
    ck(cudaSetDevice(p->opts.device), "cudaSetDevice");
    int rc = ensure_workspace(p);
    if (rc) return rc;
    std::string err;
    rc = on_stream(p, stream, [&] {
      return dm_range(p, p->ws, &p->prof, dH, dS, mu, beta, n_poles, delta_e, pole_begin, pole_end, accumulate, d_dm,
                      d_edm, d_fdm, info, &err);
    });
    return rc ? fail(p, rc, err) : PEXSI_OK;
  } catch (const CudaError& ce) {
    return map_cuda(p, ce);
  } catch (const std::bad_alloc&) {
    return fail(p, PEXSI_ERR_NOMEM, "host allocation failed");
  }
}

int pexsi_dm(pexsi_plan* p, const double* H, const double* S, double mu, double beta, int32_t n_poles, double delta_e,
             double* dm, double* edm, double* fdm, pexsi_dm_info* info) {
  return pexsi_dm_poles(p, H, S, mu, beta, n_poles, delta_e, 0, n_poles, 0, dm, edm, fdm, info);
}

int pexsi_dm_poles(pexsi_plan* p, const double* H, const double* S, double mu, double beta, int32_t n_poles,
                   double delta_e, int32_t pole_begin, int32_t pole_end, int32_t accumulate, double* dm, double* edm,
                   double* fdm, pexsi_dm_info* info) {
  if (p && p->opts.device < 0) return fail(p, PEXSI_ERR_INVALID_ARG, "host-only plan has no device");
  if (!p || !H) return fail(p, PEXSI_ERR_INVALID_ARG, "NULL plan or H");
  if (pole_begin < 0 || pole_end > n_poles || pole_begin >= pole_end)
    return fail(p, PEXSI_ERR_INVALID_ARG, "bad pole range");
  try {
    ck(cudaSetDevice(p->opts.device), "cudaSetDevice");
    int rc = ensure_workspace(p);
    if (rc) return rc;
    Workspace& ws = p->ws;
    const size_t nnz = size_t(p->sym.nnz);
    double *o_dm = ws.out, *o_edm = ws.out + nnz, *o_fdm = ws.out + 2 * nnz;
    ck(cudaMemcpyAsync(ws.H, H, sizeof(double) * nnz, cudaMemcpyHostToDevice, ws.stream), "H2D(H)");
    if (S) ck(cudaMemcpyAsync(ws.S, S, sizeof(double) * nnz, cudaMemcpyHostToDevice, ws.stream), "H2D(S)");
    if (accumulate) {
      if (dm) ck(cudaMemcpyAsync(o_dm, dm, sizeof(double) * nnz, cudaMemcpyHostToDevice, ws.stream), "H2D(dm)");
      if (edm) ck(cudaMemcpyAsync(o_edm, edm, sizeof(double) * nnz, cudaMemcpyHostToDevice, ws.stream), "H2D(edm)");
      if (fdm) ck(cudaMemcpyAsync(o_fdm, fdm, sizeof(double) * nnz, cudaMemcpyHostToDevice, ws.stream), "H2D(fdm)");
    }
    pexsi_dm_info local;
    std::string err;
    rc = dm_range(p, ws, &p->prof, ws.H, S ? ws.S : nullptr, mu, beta, n_poles, delta_e, pole_begin, pole_end,
                  accumulate, dm ? o_dm : nullptr, edm ? o_edm : nullptr, fdm ? o_fdm : nullptr, &local, &err);
    if (info) *info = local;
    if (rc) return fail(p, rc, err);
    if (dm) ck(cudaMemcpyAsync(dm, o_dm, sizeof(double) * nnz, cudaMemcpyDeviceToHost, ws.stream), "D2H(dm)");
    if (edm) ck(cudaMemcpyAsync(edm, o_edm, sizeof(double) * nnz, cudaMemcpyDeviceToHost, ws.stream), "D2H(edm)");
    if (fdm) ck(cudaMemcpyAsync(fdm, o_fdm, sizeof(double) * nnz, cudaMemcpyDeviceToHost, ws.stream), "D2H(fdm)");
    ck(cudaStreamSynchronize(ws.stream), "sync");
    return PEXSI_OK;
  } catch (const CudaError& ce) {
    return map_cuda(p, ce);
  }
}

int pexsi_selinv(pexsi_plan* p, const double* H, const double* S, double z_re, double z_im, double* ainv) {
  if (p && p->opts.device < 0) return fail(p, PEXSI_ERR_INVALID_ARG, "host-only plan has no device");
  if (!p || !H || !ainv) return fail(p, PEXSI_ERR_INVALID_ARG, "NULL argument");
  if (z_im == 0.0) return fail(p, PEXSI_ERR_INVALID_ARG, "selected inversion needs Im z != 0");
  try {
    ck(cudaSetDevice(p->opts.device), "cudaSetDevice");
    int rc = ensure_workspace(p);
    if (rc) return rc;
    Workspace& ws = p->ws;
    const size_t nnz = size_t(p->sym.nnz);
    ck(cudaMemcpyAsync(ws.H, H, sizeof(double) * nnz, cudaMemcpyHostToDevice, ws.stream), "H2D(H)");
    if (S) ck(cudaMemcpyAsync(ws.S, S, sizeof(double) * nnz, cudaMemcpyHostToDevice, ws.stream), "H2D(S)");
    if (!ws.ainv) ck(cudaMalloc(&ws.ainv, sizeof(double2) * nnz), "cudaMalloc(ainv)");
    std::string err;
    rc = selinv_one(p, ws, ws.H, S ? ws.S : nullptr, z_re, z_im, ws.ainv, &err);
    if (rc) return fail(p, rc, err);
    ck(cudaMemcpy(ainv, ws.ainv, sizeof(double2) * nnz, cudaMemcpyDeviceToHost), "D2H(ainv)");
    return PEXSI_OK;
  } catch (const CudaError& ce) {
    return map_cuda(p, ce);
  }
}

int pexsi_inertia_device(pexsi_plan* p, const double* dH, const double* dS, const double* shifts, int32_t n_shifts,
                         int64_t* counts, void* stream) {
  if (p && p->opts.device < 0) return fail(p, PEXSI_ERR_INVALID_ARG, "host-only plan has no device");
  if (!p || !dH || !shifts || !counts || n_shifts <= 0) return fail(p, PEXSI_ERR_INVALID_ARG, "bad inertia arguments");
  try {
    ck(cudaSetDevice(p->opts.device), "cudaSetDevice");
    int rc = ensure_workspace(p);
    if (rc) return rc;
    std::string err;
    rc = on_stream(p, stream, [&] { return inertia_range(p, p->ws, &p->prof, dH, dS, shifts, n_shifts, counts, &err); });
    return rc ? fail(p, rc, err) : PEXSI_OK;
  } catch (const CudaError& ce) {
    return map_cuda(p, ce);
  }
}

int pexsi_inertia(pexsi_plan* p, const double* H, const double* S, const double* shifts, int32_t n_shifts,
                  int64_t* counts) {
  if (p && p->opts.device < 0) return fail(p, PEXSI_ERR_INVALID_ARG, "host-only plan has no device");
  if (!p || !H) return fail(p, PEXSI_ERR_INVALID_ARG, "NULL plan or H");
  try {
    ck(cudaSetDevice(p->opts.device), "cudaSetDevice");
    int rc = ensure_workspace(p);
    if (rc) return rc;
    const size_t nnz = size_t(p->sym.nnz);
    ck(cudaMemcpyAsync(p->ws.H, H, sizeof(double) * nnz, cudaMemcpyHostToDevice, p->ws.stream), "H2D(H)");
    if (S) ck(cudaMemcpyAsync(p->ws.S, S, sizeof(double) * nnz, cudaMemcpyHostToDevice, p->ws.stream), "H2D(S)");
    return pexsi_inertia_device(p, p->ws.H, S ? p->ws.S : nullptr, shifts, n_shifts, counts, p->ws.stream);
  } catch (const CudaError& ce) {
    return map_cuda(p, ce);
  }
}

// ---------------------------------------------------------------- complex Hermitian H and S
namespace {
int herm_enter(pexsi_plan* p) {
  ck(cudaSetDevice(p->opts.device), "cudaSetDevice");
  int rc = ensure_workspace(p);
  if (rc) return rc;
  return hermitian_prepare(p);
}
}  // namespace

int pexsi_dm_hermitian_device(pexsi_plan* p, const double* dH, const double* dS, double mu, double beta,
                              int32_t n_poles, double delta_e, int32_t pole_begin, int32_t pole_end, int32_t accumulate,
                              double* d_dm, double* d_edm, double* d_fdm, void* stream, pexsi_dm_info* info) {
  if (p && p->opts.device < 0) return fail(p, PEXSI_ERR_INVALID_ARG, "host-only plan has no device");
  if (!p || !dH) return fail(p, PEXSI_ERR_INVALID_ARG, "NULL plan or H");
  if (pole_begin < 0 || pole_end > n_poles || pole_begin >= pole_end)
    return fail(p, PEXSI_ERR_INVALID_ARG, "bad pole range");
  try {
    int rc = herm_enter(p);
    if (rc) return rc;
    std::string err;
    rc = on_stream(p, stream, [&] {
      return dm_range_herm(p, p->ws, &p->prof, reinterpret_cast<const double2*>(dH),
                           reinterpret_cast<const double2*>(dS), mu, beta, n_poles, delta_e, pole_begin, pole_end,
                           accumulate, reinterpret_cast<double2*>(d_dm), reinterpret_cast<double2*>(d_edm),
                           reinterpret_cast<double2*>(d_fdm), info, &err);
    });
    return rc ? fail(p, rc, err) : PEXSI_OK;
  } catch (const CudaError& ce) {
    return map_cuda(p, ce);
  } catch (const std::bad_alloc&) {
    return fail(p, PEXSI_ERR_NOMEM, "host allocation failed");
  }
}

int pexsi_dm_hermitian(pexsi_plan* p, const double* H, const double* S, double mu, double beta, int32_t n_poles,
                       double delta_e, double* dm, double* edm, double* fdm, pexsi_dm_info* info) {
  if (p && p->opts.device < 0) return fail(p, PEXSI_ERR_INVALID_ARG, "host-only plan has no device");
  if (!p || !H) return fail(p, PEXSI_ERR_INVALID_ARG, "NULL plan or H");
  try {
    int rc = herm_enter(p);
    if (rc) return rc;
    Workspace& ws = p->ws;
    const size_t nnz = size_t(p->sym.nnz);
    double2 *o_dm = p->d_hout, *o_edm = p->d_hout + nnz, *o_fdm = p->d_hout + 2 * nnz;
    ck(cudaMemcpyAsync(p->d_hH, H, sizeof(double2) * nnz, cudaMemcpyHostToDevice, ws.stream), "H2D(H)");
    if (S) ck(cudaMemcpyAsync(p->d_hS, S, sizeof(double2) * nnz, cudaMemcpyHostToDevice, ws.stream), "H2D(S)");
    pexsi_dm_info local;
    std::string err;
    rc = dm_range_herm(p, ws, &p->prof, p->d_hH, S ? p->d_hS : nullptr, mu, beta, n_poles, delta_e, 0, n_poles, 0,
                       dm ? o_dm : nullptr, edm ? o_edm : nullptr, fdm ? o_fdm : nullptr, &local, &err);
    if (info) *info = local;
    if (rc) return fail(p, rc, err);
    if (dm) ck(cudaMemcpyAsync(dm, o_dm, sizeof(double2) * nnz, cudaMemcpyDeviceToHost, ws.stream), "D2H(dm)");
    if (edm) ck(cudaMemcpyAsync(edm, o_edm, sizeof(double2) * nnz, cudaMemcpyDeviceToHost, ws.stream), "D2H(edm)");
    if (fdm) ck(cudaMemcpyAsync(fdm, o_fdm, sizeof(double2) * nnz, cudaMemcpyDeviceToHost, ws.stream), "D2H(fdm)");
    ck(cudaStreamSynchronize(ws.stream), "sync");
    return PEXSI_OK;
  } catch (const CudaError& ce) {
    return map_cuda(p, ce);
  } catch (const std::bad_alloc&) {
    return fail(p, PEXSI_ERR_NOMEM, "host allocation failed");
  }
}

int pexsi_selinv_hermitian(pexsi_plan* p, const double* H, const double* S, double z_re, double z_im, double* ainv) {
  if (p && p->opts.device < 0) return fail(p, PEXSI_ERR_INVALID_ARG, "host-only plan has no device");
  if (!p || !H || !ainv) return fail(p, PEXSI_ERR_INVALID_ARG, "NULL argument");
  if (z_im == 0.0) return fail(p, PEXSI_ERR_INVALID_ARG, "selected inversion needs Im z != 0");
  try {
    int rc = herm_enter(p);
    if (rc) return rc;
    Workspace& ws = p->ws;
    const size_t nnz = size_t(p->sym.nnz);
    ck(cudaMemcpyAsync(p->d_hH, H, sizeof(double2) * nnz, cudaMemcpyHostToDevice, ws.stream), "H2D(H)");
    if (S) ck(cudaMemcpyAsync(p->d_hS, S, sizeof(double2) * nnz, cudaMemcpyHostToDevice, ws.stream), "H2D(S)");
    std::string err;
    rc = selinv_one_herm(p, ws, p->d_hH, S ? p->d_hS : nullptr, z_re, z_im, p->d_hout, &err);
    if (rc) return fail(p, rc, err);
    ck(cudaMemcpy(ainv, p->d_hout, sizeof(double2) * nnz, cudaMemcpyDeviceToHost), "D2H(ainv)");
    return PEXSI_OK;
  } catch (const CudaError& ce) {
    return map_cuda(p, ce);
  } catch (const std::bad_alloc&) {
    return fail(p, PEXSI_ERR_NOMEM, "host allocation failed");
  }
}

int pexsi_inertia_hermitian(pexsi_plan* p, const double* H, const double* S, const double* shifts, int32_t n_shifts,
                            int64_t* counts) {
  if (p && p->opts.device < 0) return fail(p, PEXSI_ERR_INVALID_ARG, "host-only plan has no device");
  if (!p || !H || !shifts || !counts || n_shifts <= 0) return fail(p, PEXSI_ERR_INVALID_ARG, "bad inertia arguments");
  try {
    int rc = herm_enter(p);
    if (rc) return rc;
    Workspace& ws = p->ws;
    const size_t nnz = size_t(p->sym.nnz);
    ck(cudaMemcpyAsync(p->d_hH, H, sizeof(double2) * nnz, cudaMemcpyHostToDevice, ws.stream), "H2D(H)");
    if (S) ck(cudaMemcpyAsync(p->d_hS, S, sizeof(double2) * nnz, cudaMemcpyHostToDevice, ws.stream), "H2D(S)");
    std::string err;
    rc = inertia_range_herm(p, ws, p->d_hH, S ? p->d_hS : nullptr, shifts, n_shifts, counts, &err);
    return rc ? fail(p, rc, err) : PEXSI_OK;
  } catch (const CudaError& ce) {
    return map_cuda(p, ce);
  } catch (const std::bad_alloc&) {
    return fail(p, PEXSI_ERR_NOMEM, "host allocation failed");
  }
}

// ---------------------------------------------------------------- groups of systems
}  // extern "C"

struct pexsi_group {
  pexsi_plan* p = nullptr;      // merged plan over all systems (owns the device memory)
  int nsys = 0;
  std::vector<int32_t> f_off;   // first merged front of each system (nsys + 1)
  int wave = 0;                 // poles per wave (0 = the workspace's batch)
  std::string fingerprint;      // key of the tuned schedule in a cache file
};

namespace {

std::string group_fingerprint(const pexsi_group* g) {
  int dev = g->p->opts.device, sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, dev);
  std::string f = "sm" + std::to_string(prop.major) + std::to_string(prop.minor) + "x" + std::to_string(sms) +
                  "/split" + std::to_string(g->p->oz_slices) + "/b" + std::to_string(g->p->b) + "/batch" +
                  std::to_string(g->p->ws.batch);
  const Symbolic& S = g->p->sym;
  for (int q = 0; q < g->nsys; ++q) {
    int64_t fe = 0, nl = 0;
    for (int32_t K = g->f_off[q]; K < g->f_off[q + 1]; ++K) {
      fe += int64_t(S.m(K)) * S.m(K);
      nl += S.s(K);
    }
    f += "/" + std::to_string(nl) + ":" + std::to_string(g->p->sys_entry_off[q + 1] - g->p->sys_entry_off[q]) + ":" +
         std::to_string(g->f_off[q + 1] - g->f_off[q]) + ":" + std::to_string(fe);
  }
  return f;
}

bool cache_lookup(const char* path, const std::string& key, int& wave, int& block, double& ms) {
  if (!path) return false;
  FILE* fh = std::fopen(path, "r");
  if (!fh) return false;
  char line[4096];
  bool found = false;
  while (std::fgets(line, sizeof(line), fh)) {
    char k[3000];
    int w = 0, b = 0;
    double t = 0;
    if (std::sscanf(line, "%2999s wave=%d block=%d ms_per_pole=%lf", k, &w, &b, &t) == 4 && key == k && w > 0 &&
        b >= 1 && b <= kOzBlockPanels) {
      wave = w;
      block = b;
      ms = t;
      found = true;  // the last entry for the key wins
    }
  }
  std::fclose(fh);
  return found;
}

}  // namespace

extern "C" {

int pexsi_group_create(const pexsi_plan* const* plans, int32_t n_plans, const pexsi_opts* opts, pexsi_group** out) {
  if (!out || !plans || n_plans <= 0) return PEXSI_ERR_INVALID_ARG;
  *out = nullptr;
  pexsi_group* g = nullptr;
  try {
    g = new pexsi_group();
    g->p = new pexsi_plan();
    pexsi_plan* p = g->p;
    int rc = init_opts(p, opts);
    if (rc == PEXSI_OK && p->opts.device < 0) rc = PEXSI_ERR_INVALID_ARG;
    std::vector<const Symbolic*> parts;
    for (int q = 0; q < n_plans && rc == PEXSI_OK; ++q) {
      if (!plans[q] || plans[q]->b != p->b) rc = PEXSI_ERR_INVALID_ARG;
      else parts.push_back(&plans[q]->sym);
    }
    if (rc) {
      delete g->p;
      delete g;
      return rc;
    }
    g->nsys = n_plans;
    p->sym = merge_symbolic(parts);
    p->flops = count_flops(p->sym, p->b);
    p->sys_entry_off.assign(1, 0);
    g->f_off.assign(1, 0);
    for (int q = 0; q < n_plans; ++q) {
      for (int64_t e : plans[q]->diag_entries) p->diag_entries.push_back(e + p->sys_entry_off.back());
      p->sys_entry_off.push_back(p->sys_entry_off.back() + plans[q]->sym.nnz);
      g->f_off.push_back(g->f_off.back() + plans[q]->sym.nsuper);
    }
    rc = upload_plan(p);
    if (rc == PEXSI_OK) rc = ensure_workspace(p);
    if (rc) {
      free_plan_device(p);
      delete p;
      delete g;
      return rc;
    }
    g->fingerprint = group_fingerprint(g);
    *out = g;
    return PEXSI_OK;
  } catch (const CudaError&) {
    if (g) { if (g->p) { free_plan_device(g->p); delete g->p; } delete g; }
    return PEXSI_ERR_CUDA;
  } catch (const std::bad_alloc&) {
    if (g) { if (g->p) { free_plan_device(g->p); delete g->p; } delete g; }
    return PEXSI_ERR_NOMEM;
  }
}

int pexsi_group_destroy(pexsi_group* g) {
  if (!g) return PEXSI_OK;
  pexsi_plan_destroy(g->p);
  delete g;
  return PEXSI_OK;
}

int pexsi_group_get_stats(const pexsi_group* g, pexsi_plan_stats* st) {
  if (!g) return PEXSI_ERR_INVALID_ARG;
  return pexsi_plan_get_stats(g->p, st);
}

int pexsi_group_get_schedule(const pexsi_group* g, pexsi_schedule* out) {
  if (!g || !out) return PEXSI_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->wave = g->wave > 0 ? g->wave : g->p->ws.batch;
  out->oz_block = g->p->oz_block;
  return PEXSI_OK;
}

int pexsi_group_set_schedule(pexsi_group* g, const pexsi_schedule* sc) {
  if (!g || !sc || sc->wave < 0 || sc->wave > g->p->ws.batch || sc->oz_block < 1 || sc->oz_block > kOzBlockPanels)
    return PEXSI_ERR_INVALID_ARG;
  g->wave = sc->wave;
  g->p->oz_block = sc->oz_block;
  return PEXSI_OK;
}

int pexsi_group_dm_device(pexsi_group* g, const double* const* dH, const double* const* dS, const double* mu,
                          const double* beta, int32_t n_poles, const double* delta_e, int32_t pole_begin,
                          int32_t pole_end, int32_t accumulate, double* const* d_dm, double* const* d_edm,
                          double* const* d_fdm, void* stream, pexsi_dm_info* info) {
  if (!g || !dH || !mu || !beta || !delta_e || !d_dm || !d_edm || !d_fdm) return PEXSI_ERR_INVALID_ARG;
  pexsi_plan* p = g->p;
  for (int q = 0; q < g->nsys; ++q)
    if (!dH[q]) return fail(p, PEXSI_ERR_INVALID_ARG, "NULL H of system " + std::to_string(q));
  if (pole_begin < 0 || pole_end > n_poles || pole_begin >= pole_end)
    return fail(p, PEXSI_ERR_INVALID_ARG, "bad pole range");
  std::vector<const double*> S(g->nsys, nullptr);
  if (dS)
    for (int q = 0; q < g->nsys; ++q) S[q] = dS[q];
  try {
    ck(cudaSetDevice(p->opts.device), "cudaSetDevice");
    std::string err;
    int rc = on_stream(p, stream, [&] {
      return dm_range_group(p, p->ws, &p->prof, g->wave, dH, S.data(), mu, beta, n_poles, delta_e, pole_begin,
                            pole_end, accumulate, d_dm, d_edm, d_fdm, info, g->f_off, &err);
    });
    return rc ? fail(p, rc, err) : PEXSI_OK;
  } catch (const CudaError& ce) {
    return map_cuda(p, ce);
  } catch (const std::bad_alloc&) {
    return fail(p, PEXSI_ERR_NOMEM, "host allocation failed");
  }
}

int pexsi_group_dm(pexsi_group* g, const double* const* H, const double* const* S, const double* mu,
                   const double* beta, int32_t n_poles, const double* delta_e, double* const* dm, double* const* edm,
                   double* const* fdm, pexsi_dm_info* info) {
  if (!g || !H || !mu || !beta || !delta_e || !dm || !edm || !fdm) return PEXSI_ERR_INVALID_ARG;
  pexsi_plan* p = g->p;
  try {
    ck(cudaSetDevice(p->opts.device), "cudaSetDevice");
    Workspace& ws = p->ws;
    const int64_t all = p->sym.nnz;
    const int n = g->nsys;
    std::vector<const double*> dH(n), dS(n, nullptr);
    std::vector<double*> o[3];
    for (int k = 0; k < 3; ++k) o[k].assign(n, nullptr);
    double* const* want[3] = {dm, edm, fdm};
    for (int q = 0; q < n; ++q) {
      if (!H[q]) return fail(p, PEXSI_ERR_INVALID_ARG, "NULL H of system " + std::to_string(q));
      const int64_t e0 = p->sys_entry_off[q], ne = p->sys_entry_off[q + 1] - e0;
      ck(cudaMemcpyAsync(ws.H + e0, H[q], sizeof(double) * ne, cudaMemcpyHostToDevice, ws.stream), "H2D(H)");
      dH[q] = ws.H + e0;
      if (S && S[q]) {
        ck(cudaMemcpyAsync(ws.S + e0, S[q], sizeof(double) * ne, cudaMemcpyHostToDevice, ws.stream), "H2D(S)");
        dS[q] = ws.S + e0;
      }
      for (int k = 0; k < 3; ++k) o[k][q] = want[k][q] ? ws.out + k * all + e0 : nullptr;
    }
    std::vector<pexsi_dm_info> local(n);
    std::string err;
    int rc = dm_range_group(p, ws, &p->prof, g->wave, dH.data(), dS.data(), mu, beta, n_poles, delta_e, 0, n_poles, 0,
                            o[0].data(), o[1].data(), o[2].data(), local.data(), g->f_off, &err);
    if (info)
      for (int q = 0; q < n; ++q) info[q] = local[q];
    if (rc) return fail(p, rc, err);
    for (int q = 0; q < n; ++q) {
      const int64_t e0 = p->sys_entry_off[q], ne = p->sys_entry_off[q + 1] - e0;
      for (int k = 0; k < 3; ++k)
        if (want[k][q])
          ck(cudaMemcpyAsync(want[k][q], ws.out + k * all + e0, sizeof(double) * ne, cudaMemcpyDeviceToHost,
                             ws.stream), "D2H");
    }
    ck(cudaStreamSynchronize(ws.stream), "sync");
    return PEXSI_OK;
  } catch (const CudaError& ce) {
    return map_cuda(p, ce);
  } catch (const std::bad_alloc&) {
    return fail(p, PEXSI_ERR_NOMEM, "host allocation failed");
  }
}

// The schedule tuner: times every candidate (wave, oz_block) on the device on
// the group's own inputs (poles [0, wave) of each system, after one untimed
// run of the first candidate), keeps the one with the least time per pole,
// and appends it to the cache file under the group's fingerprint (device,
// precision, batch capacity, the systems' sizes and front structure). A
// later call finds it there and times nothing (force = 1 re-times).
int pexsi_group_tune(pexsi_group* g, const double* const* dH, const double* const* dS, const double* mu,
                     const double* beta, int32_t n_poles, const double* delta_e, const char* cache_path,
                     int32_t force, pexsi_schedule* out) {
  if (!g || !dH || !mu || !beta || !delta_e) return PEXSI_ERR_INVALID_ARG;
  pexsi_plan* p = g->p;
  int wave = 0, block = 0;
  double ms = 0;
  if (!force && cache_lookup(cache_path, g->fingerprint, wave, block, ms) && wave <= p->ws.batch) {
    g->wave = wave;
    p->oz_block = block;
    if (out) {
      std::memset(out, 0, sizeof(*out));
      out->wave = wave;
      out->oz_block = block;
      out->ms_per_pole = ms;
      out->from_cache = 1;
    }
    return PEXSI_OK;
  }
  try {
    ck(cudaSetDevice(p->opts.device), "cudaSetDevice");
    Workspace& ws = p->ws;
    const int n = g->nsys;
    const int64_t all = p->sym.nnz;
    std::vector<const double*> S(n, nullptr);
    std::vector<double*> o[3];
    for (int k = 0; k < 3; ++k) {
      o[k].assign(n, nullptr);
      for (int q = 0; q < n; ++q) o[k][q] = ws.out + k * all + p->sys_entry_off[q];
    }
    if (dS)
      for (int q = 0; q < n; ++q) S[q] = dS[q];
    // wave candidates: the capacity, half and a quarter of it, each evened
    // out over the pole table (P = 64 at capacity 9 runs 8 waves of 8, not 7
    // of 9 and a last one of 1, which costs almost a full wave's launches)
    std::vector<int> waves;
    for (int cap = std::min(p->ws.batch, int(n_poles)); cap >= 1 && waves.size() < 3; cap /= 2) {
      const int nw = (int(n_poles) + cap - 1) / cap, w = (int(n_poles) + nw - 1) / nw;
      if (std::find(waves.begin(), waves.end(), w) == waves.end()) waves.push_back(w);
      if (cap == 1) break;
    }
    std::vector<int> blocks = p->oz_slices > 0 ? std::vector<int>{4, 2, 1} : std::vector<int>{p->oz_block};
    std::vector<pexsi_dm_info> info(n);
    std::string err;
    double best = 1e300;
    int bw = waves[0], bb = blocks[0], cands = 0;
    bool warmed = false;
    for (int w : waves)
      for (int blk : blocks) {
        p->oz_block = blk;
        for (int rep = warmed ? 0 : 1; rep >= 0; --rep) {  // one untimed run before the first timing
          int rc = dm_range_group(p, ws, nullptr, w, dH, S.data(), mu, beta, n_poles, delta_e, 0, w, 0, o[0].data(),
                                  o[1].data(), o[2].data(), info.data(), g->f_off, &err);
          if (rc) return fail(p, rc, err);
        }
        warmed = true;
        ++cands;
        const double per = info[0].ms_total / w;
        if (per < best) {
          best = per;
          bw = w;
          bb = blk;
        }
      }
    g->wave = bw;
    p->oz_block = bb;
    if (cache_path) {
      FILE* fh = std::fopen(cache_path, "a");
      if (fh) {
        std::fprintf(fh, "%s wave=%d block=%d ms_per_pole=%.6f\n", g->fingerprint.c_str(), bw, bb, best);
        std::fclose(fh);
      }
    }
    if (out) {
      std::memset(out, 0, sizeof(*out));
      out->wave = bw;
      out->oz_block = bb;
      out->ms_per_pole = best;
      out->candidates = cands;
    }
    return PEXSI_OK;
  } catch (const CudaError& ce) {
    return map_cuda(p, ce);
  } catch (const std::bad_alloc&) {
    return fail(p, PEXSI_ERR_NOMEM, "host allocation failed");
  }
}

const char* pexsi_group_last_error_detail(const pexsi_group* g) { return g ? g->p->last_error.c_str() : ""; }

}  // extern "C"
