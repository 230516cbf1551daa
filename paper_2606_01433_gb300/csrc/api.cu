// C ABI of libgdsw.so and the orchestration of set-up and apply
// (arXiv 2606.01433: Section 2.1 two-level monolithic GDSW, Section 2.2 multilevel
// recursion and four-level preconditioner, Section 3 FGMRES).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <tuple>

#include "common.h"
#include "kernels.h"
#include "setup.h"

namespace gdsw {

void fgmres_solve(gdsw_ctx* c, const double* b, double* x, gdsw_solve_info* info);

static thread_local std::string g_setup_error;

static double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

std::atomic<int64_t>& launch_counter() {
  static std::atomic<int64_t> n{0};
  return n;
}

// ------------------------------------------------------------------ profiling helpers
static void prof_collect(gdsw_ctx* c) {
  for (auto& p : c->pending) {
    cudaEventSynchronize(p.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    c->prof.calls[p.group] += 1;
    c->prof.ms[p.group] += ms;
    c->prof.bytes[p.group] += p.bytes;
    c->ev_pool.push_back(p.a);
    c->ev_pool.push_back(p.b);
  }
  c->pending.clear();
}

// ------------------------------------------------------------------ device views
struct SlabDevice {
  SlabView v{};
  std::vector<int32_t> owner;
  std::vector<int32_t> part_of_row;
};

static SlabView upload_slabview(DevArena& A, const SlabSet& S, cudaStream_t s, std::vector<int32_t>* owner_out) {
  std::vector<int32_t> owner(S.nvec), pslab(S.nvec), pidx(S.nvec), slab_base(S.nsub + 1);
  std::vector<int64_t> fS, fG, fW;
  std::vector<int32_t> ldS, ldG, ldW, m;
  int sb = 0;
  for (int i = 0; i < S.nsub; ++i) {
    slab_base[i] = sb;
    for (int k = 0; k < S.K[i]; ++k) {
      fS.push_back(S.fS[i][k]); fG.push_back(S.fG[i][k]); fW.push_back(S.fW[i][k]);
      ldS.push_back(S.ldS[i][k]); ldG.push_back(S.ldG[i][k]); ldW.push_back(S.ldW[i][k]);
      m.push_back(S.m[i][k]);
      int64_t p0 = S.voff[i] + S.soff[i][k];
      for (int r = 0; r < S.s[i][k]; ++r) {
        owner[p0 + r] = i;
        pslab[p0 + r] = k;
        pidx[p0 + r] = r;
      }
    }
    sb += S.K[i];
  }
  slab_base[S.nsub] = sb;
  SlabView v;
  v.nvec = S.nvec;
  v.gdof = A.upload(S.gdof, s);
  v.owner = A.upload(owner, s);
  v.pslab = A.upload(pslab, s);
  v.pidx = A.upload(pidx, s);
  v.voff = A.upload(S.voff, s);
  v.slab_base = A.upload(slab_base, s);
  v.fS = A.upload(fS, s); v.fG = A.upload(fG, s); v.fW = A.upload(fW, s);
  v.ldS = A.upload(ldS, s); v.ldG = A.upload(ldG, s); v.ldW = A.upload(ldW, s);
  v.m = A.upload(m, s);
  if (owner_out) *owner_out = owner;
  return v;
}

static MatView matview(const gdsw_ctx* c) {
  MatView v;
  v.n = c->mesh.n;
  v.nu = c->mesh.nu;
  v.a_ptr = c->d_a_ptr; v.a_col = c->d_a_col;
  v.bt_ptr = c->d_bt_ptr; v.bt_col = c->d_bt_col;
  v.b_ptr = c->d_b_ptr; v.b_col = c->d_b_col;
  v.aval = c->d_val;
  v.btval = c->d_val + 9 * c->nnzb;
  v.bval = v.btval + 3 * c->nbt;
  return v;
}

template <typename T>
static T* ptr_at(void* base, int64_t off) {
  return static_cast<T*>(base) + off;
}

// ------------------------------------------------------------------ block-tridiagonal LDL^T factorisation
// For slab blocks A_kk (diagonal) and B_k (rows of slab k coupled to slab k-1; the operator is
// symmetric, so the block above the diagonal is B_k^T), compute in place
//   S_0 = A_00, S_k = A_kk - G_k B_k^T,  G_k = B_k S_{k-1}^{-1},  Sinv_k = S_k^{-1},
// so that A = L D L^T with L_{k,k-1} = G_k and D = diag(S_k).
template <typename T>
static void factor_slabs(const SlabSet& S, T* fac, double& minpiv, cudaStream_t s) {
  DevArena tmp(s);
  int64_t maxB = 1, maxC = 1;
  for (int k = 0; k < S.Kmax; ++k) {
    int64_t sb = 0, sc = 0;
    for (int i = 0; i < S.nsub; ++i)
      if (k >= 1 && k < S.K[i]) sb += int64_t(S.m[i][k]) * S.ldG[i][k];
    maxB = std::max(maxB, sb);
    (void)sc;
  }
  T* scrB = tmp.alloc<T>(maxB);
  minpiv = 1e300;
  try {
    // symmetric block LDL^T: G_k = B_k S_{k-1}^{-1}, S_k = A_kk - G_k B_k^T
    for (int k = 0; k < S.Kmax; ++k) {
      if (k >= 1) {
        std::vector<GemmTaskP> tg, tu;
        int64_t off = 0;
        for (int i = 0; i < S.nsub; ++i) {
          if (k >= S.K[i] || S.m[i][k] == 0) continue;
          int m = S.m[i][k], sp = S.s[i][k - 1];
          int64_t cnt = int64_t(m) * S.ldG[i][k];
          GDSW_CUDA(cudaMemcpyAsync(scrB + off, fac + S.fG[i][k], cnt * sizeof(T), cudaMemcpyDeviceToDevice, s));
          tg.push_back({scrB + off, fac + S.fS[i][k - 1], fac + S.fG[i][k], m, sp, sp, S.ldG[i][k], S.ldS[i][k - 1],
                        S.ldG[i][k], 0, 0, 1.0, 0.0});
          tu.push_back({fac + S.fG[i][k], scrB + off, fac + S.fS[i][k], m, m, sp, S.ldG[i][k], S.ldG[i][k],
                        S.ldS[i][k], 0, 1, -1.0, 1.0});
          off += cnt;
        }
        run_gemm<T>(tmp, tg, s);
        run_gemm<T>(tmp, tu, s);
      }
      std::vector<InvTaskP> inv;
      for (int i = 0; i < S.nsub; ++i)
        if (k < S.K[i]) inv.push_back({fac + S.fS[i][k], S.s[i][k], S.ldS[i][k], 0});
      std::vector<double> mp;
      run_inverse<T>(tmp, inv, mp, s);
      for (double v : mp) minpiv = std::min(minpiv, v);
    }
    GDSW_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    tmp.free_all();
    throw;
  }
  tmp.free_all();
}

// multi right-hand-side solve with the LDU factors: R (rows in slab order, ld ldt per
// part) holds the right-hand sides and is overwritten by the forward sweep; W receives the
// solution.
template <typename T>
static void sweep_multi(const SlabSet& S, const T* fac, T* R, T* W, const std::vector<int64_t>& toff,
                        const std::vector<int>& ldt, const std::vector<int>& nc, cudaStream_t s) {
  DevArena tmp(s);
  try {
    for (int k = 0; k < S.Kmax; ++k) {
      std::vector<GemmTaskP> g, d;
      for (int i = 0; i < S.nsub; ++i) {
        if (k >= S.K[i] || nc[i] == 0) continue;
        T* Rk = R + toff[i] + S.soff[i][k] * ldt[i];
        if (k >= 1 && S.m[i][k] > 0)
          g.push_back({fac + S.fG[i][k], R + toff[i] + S.soff[i][k - 1] * ldt[i], Rk, S.m[i][k], nc[i], S.s[i][k - 1],
                       S.ldG[i][k], ldt[i], ldt[i], 0, 0, -1.0, 1.0});
        d.push_back({fac + S.fS[i][k], Rk, W + toff[i] + S.soff[i][k] * ldt[i], S.s[i][k], nc[i], S.s[i][k],
                     S.ldS[i][k], ldt[i], ldt[i], 0, 0, 1.0, 0.0});
      }
      run_gemm<T>(tmp, g, s);
      run_gemm<T>(tmp, d, s);
    }
    for (int j = 0; j + 1 < S.Kmax; ++j) {
      std::vector<GemmTaskP> b;
      for (int i = 0; i < S.nsub; ++i) {
        int k = S.K[i] - 2 - j;
        if (k < 0 || nc[i] == 0 || S.m[i][k + 1] == 0) continue;
        // X_k -= G_{k+1}^T X_{k+1}[0:m_{k+1}]  (the super-diagonal block of the symmetric LDL^T)
        b.push_back({fac + S.fG[i][k + 1], W + toff[i] + S.soff[i][k + 1] * ldt[i], W + toff[i] + S.soff[i][k] * ldt[i],
                     S.s[i][k], nc[i], S.m[i][k + 1], S.ldG[i][k + 1], ldt[i], ldt[i], 1, 0, -1.0, 1.0});
      }
      run_gemm<T>(tmp, b, s);
    }
    GDSW_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    tmp.free_all();
    throw;
  }
  tmp.free_all();
}

// ------------------------------------------------------------------ apply plans
static void finish_plan(DevArena& A, GemvPlan& P, std::vector<GemvTask>& tasks, std::vector<GemvTile>& tiles,
                        cudaStream_t s) {
  P.d_tasks = A.upload(tasks, s);
  P.d_tiles = A.upload(tiles, s);
}

static void add_task(std::vector<GemvTask>& tasks, std::vector<GemvTile>& tiles, const GemvTask& t, int rpt) {
  if (t.rows <= 0) return;
  int id = int(tasks.size());
  tasks.push_back(t);
  for (int r = 0; r < t.rows; r += rpt) tiles.push_back({id, r});
}

// algorithmic bytes of the tasks [t0, t1): matrix entries read once, input read once, output
// written (plus read when accumulated)
static double plan_bytes(const std::vector<GemvTask>& tasks, int t0, int t1, size_t esz, size_t vsz,
                         bool transposed = false) {
  double b = 0;
  for (int t = t0; t < t1; ++t) {
    const GemvTask& q = tasks[t];
    if (q.kind == 1) {  // the symmetric block's distinct entries, input once, partials written
      const double s = q.rows, T = double(q.cols) / q.ld;
      b += s * (s + 1) / 2 * esz + s * vsz + double(q.ld) * q.ld * T * vsz;
      continue;
    }
    double in = transposed ? q.rows : q.cols, out = transposed ? q.cols : q.rows;
    b += double(q.rows) * q.cols * esz + in * vsz + out * vsz * (q.base >= 0 ? 2 : 1);
  }
  return b;
}

// Work list of the persistent sweep (same tasks and tiles as the per-step launches).  Per
// flattened slab q four counters: Y (tiles of the G task that writes y_q), P (symmetric
// tiles of S_q^{-1}), W (tiles that write w_q: dense S_q^{-1} rows or reductions), X
// (backward tiles that write x_q).  Every item is listed after all producers it waits for.
struct TaskRec {
  int task, q, step, role, t0, t1;  // role: 0 dense S^{-1}, 1 symmetric S^{-1}, 2 G, 3 reduction, 4 backward
};

static void build_sweep(gdsw_ctx* c, LevelDev& L, int nslab, int Kmax, const std::vector<GemvTask>& tasks,
                        const std::vector<GemvTile>& tiles, const std::vector<GemvTask>& rtasks,
                        const std::vector<GemvTile>& rtiles, const std::vector<TaskRec>& recs, int xs_elems) {
  auto ctr = [](int q, int kind) { return 1 + 4 * q + kind; };
  enum { Y = 0, P = 1, W = 2, X = 3 };
  const int nctr = 1 + 4 * nslab;
  std::vector<int> nsig(nctr, 0), last(nctr, -1);
  std::vector<SweepItem> items;
  const int roff = int(tasks.size());
  auto emit = [&](int op, int task, int arg, int signal, int w0, int w1) {
    SweepItem it{op, task, arg, signal, -1, 0, -1, 0};
    const int idx = int(items.size());
    if (w0 >= 0 && nsig[w0] > 0) {
      GDSW_CHECK(last[w0] < idx, GDSW_ERR_INVALID_ARG, "sweep list: producer after consumer");
      it.wait0 = w0;
      it.need0 = nsig[w0];
    }
    if (w1 >= 0 && nsig[w1] > 0) {
      GDSW_CHECK(last[w1] < idx, GDSW_ERR_INVALID_ARG, "sweep list: producer after consumer");
      it.wait1 = w1;
      it.need1 = nsig[w1];
    }
    items.push_back(it);
    if (signal >= 0) {
      ++nsig[signal];
      last[signal] = idx;
    }
  };
  auto emit_reduce = [&](int step) {
    for (const TaskRec& r : recs)
      if (r.role == 3 && r.step == step)
        for (int t = r.t0; t < r.t1; ++t) emit(SWEEP_REDUCE, roff + r.task, rtiles[t].row0, ctr(r.q, W), ctr(r.q, P), -1);
  };
  for (int k = 0; k < Kmax; ++k) {
    for (const TaskRec& r : recs) {
      if (r.step != k || r.role > 2) continue;
      const int wy = k > 0 ? ctr(r.q, Y) : -1;  // y_q is final once the G task of step k-1 is done
      const int sig = r.role == 0 ? ctr(r.q, W) : (r.role == 1 ? ctr(r.q, P) : ctr(r.q + 1, Y));
      for (int t = r.t0; t < r.t1; ++t) emit(r.role == 1 ? SWEEP_SYM : SWEEP_ROWS, r.task, tiles[t].row0, sig, wy, -1);
    }
    if (k > 0) emit_reduce(k - 1);  // one step behind, so that the partials are mostly done
  }
  if (Kmax > 0) emit_reduce(Kmax - 1);
  for (const TaskRec& r : recs) {  // backward, in step order: x_k = w_k - G_{k+1}^T x_{k+1}
    if (r.role != 4) continue;
    const int wx = nsig[ctr(r.q + 1, X)] > 0 ? ctr(r.q + 1, X) : ctr(r.q + 1, W);
    for (int t = r.t0; t < r.t1; ++t) emit(SWEEP_COLS, r.task, tiles[t].row0, ctr(r.q, X), ctr(r.q, W), wx);
  }
  std::vector<GemvTask> all = tasks;
  all.insert(all.end(), rtasks.begin(), rtasks.end());
  SweepPlan& SP = L.sweep;
  SP.nitems = int(items.size());
  SP.nctr = nctr;
  SP.xs_elems = (xs_elems + 3) & ~3;
  SP.d_items = c->arena.upload(items, c->stream);
  SP.d_tasks = c->arena.upload(all, c->stream);
  SP.d_ctr = c->arena.alloc<unsigned>(nctr);
  SP.G = L.fwd.rows_per_tile / 32;
}

static void resize_sweep(LevelDev& L, int ctas_per_sm) {
  if (L.sweep.nitems == 0) return;
  L.sweep.ctas_per_sm = ctas_per_sm;
  if (L.prec == GDSW_FP64)
    size_sweep<double, double>(L.sweep);
  else if (L.prec == GDSW_FP32)
    size_sweep<float, float>(L.sweep);
  else
    size_sweep<__nv_bfloat16, float>(L.sweep);
}

static void build_local_plan(gdsw_ctx* c, const SlabSet& S, LevelDev& L) {
  std::vector<GemvTask> tasks;
  std::vector<GemvTile> tiles;
  std::vector<GemvTask> rtasks;  // reductions of the symmetric partial sums
  std::vector<GemvTile> rtiles;
  std::vector<TaskRec> recs;
  const size_t esz = elem_size(L.prec), vsz = L.prec == GDSW_FP64 ? 8 : 4;
  const int rpt = L.fwd.rows_per_tile;
  const int64_t nv = S.nvec;
  const int TT = L.sym_T;
  std::vector<int> sb(S.nsub + 1, 0);  // first flattened slab index of each part
  for (int i = 0; i < S.nsub; ++i) sb[i + 1] = sb[i] + S.K[i];
  int64_t part_off = 2 * nv;          // partial sums live behind the two local vectors
  int xs_elems = 8;                   // shared staging of the persistent sweep
  L.fwd.launch_task_off = {0};
  L.fwd.launch_tile_off = {0};
  L.fwd_ld.clear();
  for (int k = 0; k < S.Kmax; ++k) {
    int mld = 8;
    for (int i = 0; i < S.nsub; ++i) {
      if (k >= S.K[i]) continue;
      const int q = sb[i] + k;
      int64_t y = S.voff[i] + S.soff[i][k];
      const int sk = S.s[i][k];
      if (L.psym[q]) {
        const int nt = (sk + TT - 1) / TT;
        GemvTask t{L.pS[q], y, nv + y, -1, sk, nt * TT, nt, 1.0f, 1, 0, part_off};
        int id = int(tasks.size());
        tasks.push_back(t);
        const int t0 = int(tiles.size());
        for (int I = 0; I < nt; ++I)
          for (int J = I; J < nt; ++J) tiles.push_back({id, (I << 16) | J});
        recs.push_back({id, q, k, 1, t0, int(tiles.size())});
        int rid = int(rtasks.size());
        rtasks.push_back(t);
        const int r0t = int(rtiles.size());
        for (int r0 = 0; r0 < sk; r0 += 256) rtiles.push_back({rid, r0});
        recs.push_back({rid, q, k, 3, r0t, int(rtiles.size())});
        part_off += int64_t(nt) * nt * TT;
        mld = std::max(mld, 11 * TT);
      } else {
        GemvTask t{L.pS[q], y, nv + y, -1, sk, sk, S.ldS[i][k], 1.0f};
        const int t0 = int(tiles.size());
        add_task(tasks, tiles, t, rpt);
        if (int(tiles.size()) > t0) recs.push_back({int(tasks.size()) - 1, q, k, 0, t0, int(tiles.size())});
        mld = std::max(mld, S.ldS[i][k]);
      }
      if (k + 1 < S.K[i] && S.m[i][k + 1] > 0) {
        int64_t y1 = S.voff[i] + S.soff[i][k + 1];
        GemvTask g{L.pG[q + 1], y, y1, y1, S.m[i][k + 1], sk, S.ldG[i][k + 1], -1.0f};
        const int t0 = int(tiles.size());
        add_task(tasks, tiles, g, rpt);
        if (int(tiles.size()) > t0) recs.push_back({int(tasks.size()) - 1, q, k, 2, t0, int(tiles.size())});
        mld = std::max(mld, S.ldG[i][k + 1]);
      }
    }
    L.fwd.launch_task_off.push_back(int(tasks.size()));
    L.fwd.launch_tile_off.push_back(int(tiles.size()));
    L.fwd_ld.push_back(mld);
    xs_elems = std::max(xs_elems, mld);
  }
  L.npart = part_off - 2 * nv;
  L.red.launch_task_off = {0, int(rtasks.size())};
  L.red.launch_tile_off = {0, int(rtiles.size())};
  L.red_bytes = 0;
  for (const GemvTask& t : rtasks) L.red_bytes += (double(t.ld) * t.ld * TT + t.rows) * vsz;
  finish_plan(c->arena, L.red, rtasks, rtiles, c->stream);
  // backward: x_k = w_k - G_{k+1}^T x_{k+1}[0:m_{k+1}], transposed GEMV over column tiles
  L.bwd.transposed = true;
  L.bwd.launch_task_off = {int(tasks.size())};
  L.bwd.launch_tile_off = {int(tiles.size())};
  L.bwd_ld.clear();
  for (int j = 0; j + 1 < S.Kmax; ++j) {
    int mrows = 8;
    for (int i = 0; i < S.nsub; ++i) {
      int k = S.K[i] - 2 - j;
      if (k < 0 || S.m[i][k + 1] == 0) continue;
      int64_t y = nv + S.voff[i] + S.soff[i][k];
      int64_t x = nv + S.voff[i] + S.soff[i][k + 1];
      GemvTask t{L.pG[sb[i] + k + 1], x, y, y, S.m[i][k + 1], S.s[i][k], S.ldG[i][k + 1], -1.0f};
      int id = int(tasks.size());
      tasks.push_back(t);
      const int t0 = int(tiles.size());
      for (int c0 = 0; c0 < t.cols; c0 += gemvt_tile_cols(L.prec)) tiles.push_back({id, c0});
      recs.push_back({id, sb[i] + k, S.Kmax + j, 4, t0, int(tiles.size())});
      mrows = std::max(mrows, t.rows);
    }
    L.bwd.launch_task_off.push_back(int(tasks.size()));
    L.bwd.launch_tile_off.push_back(int(tiles.size()));
    L.bwd_ld.push_back(mrows);
    xs_elems = std::max(xs_elems, mrows);
  }
  L.fwd_bytes.clear();
  L.bwd_bytes.clear();
  for (int k = 0; k < L.fwd.nlaunch(); ++k)
    L.fwd_bytes.push_back(plan_bytes(tasks, L.fwd.launch_task_off[k], L.fwd.launch_task_off[k + 1], esz, vsz));
  for (int k = 0; k < L.bwd.nlaunch(); ++k)
    L.bwd_bytes.push_back(plan_bytes(tasks, L.bwd.launch_task_off[k], L.bwd.launch_task_off[k + 1], esz, vsz, true));
  build_sweep(c, L, sb[S.nsub], S.Kmax, tasks, tiles, rtasks, rtiles, recs, xs_elems);
  resize_sweep(L, L.sweep.ctas_per_sm);
  GemvTask* dt = c->arena.upload(tasks, c->stream);
  GemvTile* dl = c->arena.upload(tiles, c->stream);
  L.fwd.d_tasks = dt;
  L.fwd.d_tiles = dl;
  L.bwd.d_tasks = dt;
  L.bwd.d_tiles = dl;
}

// Tile-shape autotuner for the level-1 local solves, run at the end of the set-up: whole
// preconditioner applies (level-1 sweeps with the coarse branch running beside them on the
// second stream) are timed with CUDA events, best of three after a warm-up, with 32, 64 and
// 128 rows per forward tile, each as one launch per slab step and as the persistent launch;
// the fastest is kept.  Every candidate computes the same numbers bit for bit -- a row's dot
// product is one warp's in a fixed order and the persistent launch runs the same tiles -- so
// the choice changes only the schedule.  Small problems (level-1 sweeps under 64 MB) keep
// the defaults.
static void apply_precond_impl(gdsw_ctx* c, const double* r, double* z, cudaStream_t s);

static void autotune_level1(gdsw_ctx* c) {
  LevelDev& L = c->ld[0];
  double bytes = L.red_bytes;
  for (double b : L.fwd_bytes) bytes += b;
  for (double b : L.bwd_bytes) bytes += b;
  if (bytes < 64e6 || L.n <= 0) return;
  cudaStream_t s = c->stream;
  DevArena tmp(s);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  try {
    const int64_t n = c->mesh.n;
    double* r = tmp.alloc<double>(n);
    double* z = tmp.alloc<double>(n);
    GDSW_CUDA(cudaMemsetAsync(r, 0, sizeof(double) * n, s));
    GDSW_CUDA(cudaEventCreate(&e0));
    GDSW_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int bestG = 1, curG = L.fwd.rows_per_tile / 32;
    bool bestP = false;
    for (int G : {1, 2, 4}) {
      if (G != curG) {
        L.fwd.rows_per_tile = 32 * G;
        build_local_plan(c, c->lh[0].loc, L);
        curG = G;
      }
      for (bool P : {false, true}) {
        L.persistent = P;
        apply_precond_impl(c, r, z, s);
        float t = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
          GDSW_CUDA(cudaEventRecord(e0, s));
          apply_precond_impl(c, r, z, s);
          GDSW_CUDA(cudaEventRecord(e1, s));
          GDSW_CUDA(cudaEventSynchronize(e1));
          float ms = 0.f;
          GDSW_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          t = std::min(t, ms);
        }
        if (t < best) {
          best = t;
          bestG = G;
          bestP = P;
        }
      }
    }
    if (bestG != curG) {
      L.fwd.rows_per_tile = 32 * bestG;
      build_local_plan(c, c->lh[0].loc, L);
    }
    L.persistent = bestP;
    L.tuned_ms = best;
  } catch (...) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    tmp.free_all();
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  tmp.free_all();
}

// ------------------------------------------------------------------ coarse space upload
struct CSBuild {
  std::vector<int64_t> toff;   // per part offset of the n_I x ldt interior blocks
  std::vector<int> ldt, nc;
  int64_t ttot = 0;
  std::vector<int32_t> part_of_irow;
};

static CSBuild cs_layout(const CoarseSpace& C) {
  CSBuild b;
  b.toff.assign(C.nparts + 1, 0);
  for (int J = 0; J < C.nparts; ++J) {
    int c = int(C.coff[J + 1] - C.coff[J]);
    int64_t nI = C.ioff[J + 1] - C.ioff[J];
    b.nc.push_back(c);
    b.ldt.push_back(int(pad8(std::max(c, 1))));
    b.toff[J + 1] = b.toff[J] + nI * b.ldt[J];
    for (int64_t r = 0; r < nI; ++r) b.part_of_irow.push_back(J);
  }
  b.ttot = b.toff[C.nparts];
  return b;
}

// upload the apply-side coarse-space data (interior lists, columns, PhiT layout, plans)
static void upload_coarse_space(gdsw_ctx* c, int l, int phi_prec) {
  const CoarseSpace& C = c->lh[l].cs;
  LevelDev& L = c->ld[l];
  cudaStream_t s = c->stream;
  L.n0 = C.n0;
  L.phi_prec = phi_prec;
  if (C.n0 == 0) return;
  L.idofs = c->arena.upload(C.idofs, s);
  L.cols = c->arena.upload(C.cols, s);
  L.gdofs = c->arena.upload(C.gdofs, s);
  L.gcol = c->arena.upload(C.gcol, s);
  L.nidofs = int64_t(C.idofs.size());
  L.ncols = int64_t(C.cols.size());
  L.ngamma = int64_t(C.gdofs.size());
  L.rr_ptr = c->arena.upload(C.rr_ptr, s);
  L.rr_pos = c->arena.upload(C.rr_pos, s);
  L.rg_ptr = c->arena.upload(C.rg_ptr, s);
  L.rg_dof = c->arena.upload(C.rg_dof, s);
  L.rg_val = c->arena.upload(C.rg_val, s);
  L.gval = c->arena.upload(C.gval, s);
  L.gu_dof = c->arena.upload(C.gu_dof, s);
  L.gu_ptr = c->arena.upload(C.gu_ptr, s);
  L.ngu = int64_t(C.gu_dof.size());
  // PhiT layout: part J stores c_J rows of length pad8(n_IJ)
  // 256-dof tiles of every part's interior, shared by the prolongation and the restriction
  std::vector<ProMeta> meta(C.nparts);
  std::vector<int32_t> tp, tc, tr, pnt(C.nparts, 0), qcnt(C.cols.size(), 0);
  std::vector<int64_t> poff(C.nparts + 1, 0), qst(C.cols.size(), 0);
  int64_t off = 0;
  L.max_c = 1;
  for (int J = 0; J < C.nparts; ++J) {
    int cJ = int(C.coff[J + 1] - C.coff[J]);
    int nI = int(C.ioff[J + 1] - C.ioff[J]);
    int ld = int(pad8(std::max(nI, 1)));
    meta[J] = {off, C.ioff[J], C.coff[J], ld, nI, cJ, 0};
    if (cJ > 0 && nI > 0)
      for (int col0 = 0; col0 < nI; col0 += 256) {
        tp.push_back(J);
        tc.push_back(col0);
        tr.push_back(pnt[J]++);
      }
    poff[J + 1] = poff[J] + int64_t(cJ) * pnt[J];
    for (int j = 0; j < cJ; ++j) {
      qst[C.coff[J] + j] = poff[J] + int64_t(j) * pnt[J];
      qcnt[C.coff[J] + j] = pnt[J];
    }
    L.max_c = std::max(L.max_c, cJ);
    off += int64_t(cJ) * ld;
  }
  L.pro_meta = reinterpret_cast<int64_t*>(c->arena.upload(meta, s));
  L.pro_tile_part = c->arena.upload(tp, s);
  L.pro_tile_col0 = c->arena.upload(tc, s);
  L.pro_tile_rank = c->arena.upload(tr, s);
  L.n_pro_tiles = int(tp.size());
  L.part_poff = c->arena.upload(poff, s);
  L.part_ntiles = c->arena.upload(pnt, s);
  L.q_start = c->arena.upload(qst, s);
  L.q_count = c->arena.upload(qcnt, s);
  L.partial = c->arena.alloc<double>(size_t(std::max<int64_t>(poff[C.nparts], 1)));
  GDSW_CHECK(8 * (256 + 33 * int64_t(L.max_c)) <= 200 * 1024, GDSW_ERR_INVALID_ARG,
             "a part has too many coarse columns for the restriction tile");
  L.phiT = c->arena.alloc<char>(size_t(std::max<int64_t>(off, 1)) * elem_size(phi_prec));
  GDSW_CUDA(cudaMemsetAsync(L.phiT, 0, size_t(std::max<int64_t>(off, 1)) * elem_size(phi_prec), s));
  L.r0 = c->arena.alloc<double>(C.n0);
  L.x0 = c->arena.alloc<double>(C.n0);
}

static std::vector<int64_t> phi_offsets(const CoarseSpace& C, std::vector<int32_t>& ld) {
  std::vector<int64_t> off(C.nparts + 1, 0);
  ld.resize(C.nparts);
  for (int J = 0; J < C.nparts; ++J) {
    int cJ = int(C.coff[J + 1] - C.coff[J]);
    int nI = int(C.ioff[J + 1] - C.ioff[J]);
    ld[J] = int(pad8(std::max(nI, 1)));
    off[J + 1] = off[J] + int64_t(cJ) * ld[J];
  }
  return off;
}

// segment lists for A0 = sum of keyed contributions, built on the host
struct SegList {
  std::vector<int64_t> key, ptr, pos;
  std::vector<double> w;  // per entry weight (empty: all 1)
};
static SegList make_segments(std::vector<std::pair<int64_t, int64_t>>& kv) {
  std::stable_sort(kv.begin(), kv.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
  SegList L;
  L.ptr.push_back(0);
  for (size_t q = 0; q < kv.size(); ++q) {
    if (q == 0 || kv[q].first != kv[q - 1].first) {
      if (q > 0) L.ptr.push_back(int64_t(q));
      L.key.push_back(kv[q].first);
    }
    L.pos.push_back(kv[q].second);
  }
  if (!kv.empty()) L.ptr.push_back(int64_t(kv.size()));
  return L;
}

// the same with a weight per entry: kvw = (key, source position, weight)
static SegList make_segments_w(std::vector<std::tuple<int64_t, int64_t, double>>& kvw) {
  std::stable_sort(kvw.begin(), kvw.end(),
                   [](const auto& a, const auto& b) { return std::get<0>(a) < std::get<0>(b); });
  SegList L;
  L.ptr.push_back(0);
  for (size_t q = 0; q < kvw.size(); ++q) {
    if (q == 0 || std::get<0>(kvw[q]) != std::get<0>(kvw[q - 1])) {
      if (q > 0) L.ptr.push_back(int64_t(q));
      L.key.push_back(std::get<0>(kvw[q]));
    }
    L.pos.push_back(std::get<1>(kvw[q]));
    L.w.push_back(std::get<2>(kvw[q]));
  }
  if (!kvw.empty()) L.ptr.push_back(int64_t(kvw.size()));
  return L;
}

static void run_segments(gdsw_ctx* c, SegList& L, const double* src, double* dst, DevArena& tmp) {
  if (L.key.empty()) return;
  int64_t* k = tmp.upload(L.key, c->stream);
  int64_t* p = tmp.upload(L.ptr, c->stream);
  int64_t* q = tmp.upload(L.pos, c->stream);
  double* w = L.w.empty() ? nullptr : tmp.upload(L.w, c->stream);
  segsum(k, p, q, w, int64_t(L.key.size()), src, dst, c->stream);
}

// ------------------------------------------------------------------ factor storage
// Final storage of a level's factors in the apply precision.  FP32/BF16 diagonal inverses
// S_k^{-1} of at least 4 tiles per side are kept as their upper-triangle T x T tiles (the
// block is symmetric up to rounding: the operator is, and the inverse of a symmetric matrix
// is), the others densely; the G_k blocks follow each slab's S_k^{-1}.
template <typename T>
static void store_factors(gdsw_ctx* c, const SlabSet& S, const T* fac, LevelDev& L, int prec, DevArena& tmp) {
  cudaStream_t s = c->stream;
  const int TT = sym_tile_size(prec);
  L.prec = prec;
  L.nvec = S.nvec;
  L.sym_T = TT;
  L.pS.clear();
  L.pG.clear();
  L.psym.clear();
  std::vector<PackTile> tiles;
  int64_t off = 0;
  for (int i = 0; i < S.nsub; ++i)
    for (int k = 0; k < S.K[i]; ++k) {
      const int sk = S.s[i][k];
      // FP64 stays dense: on GB300 the FP64 sweep is bound by FP64 FMAs, which packing
      // does not reduce (each stored entry then feeds two products)
      const bool sym = prec != GDSW_FP64 && sk >= 4 * TT;
      L.psym.push_back(sym);
      L.pS.push_back(off);
      if (sym) {
        const int nt = (sk + TT - 1) / TT;
        for (int I = 0; I < nt; ++I)
          for (int J = I; J < nt; ++J) {
            tiles.push_back({S.fS[i][k] + int64_t(I) * TT * S.ldS[i][k] + int64_t(J) * TT, off, S.ldS[i][k],
                             std::min(TT, sk - I * TT), std::min(TT, sk - J * TT), 0});
            off += int64_t(TT) * TT;
          }
      } else {
        off += int64_t(sk) * S.ldS[i][k];
      }
      L.pG.push_back(off);
      if (k > 0) off += int64_t(S.m[i][k]) * S.ldG[i][k];
    }
  L.nfac = off;
  T* packed = tmp.alloc<T>(std::max<int64_t>(off, 1));
  GDSW_CUDA(cudaMemsetAsync(packed, 0, sizeof(T) * std::max<int64_t>(off, 1), s));
  pack_tiles<T>(tmp, fac, packed, tiles, TT, s);
  size_t q = 0;
  for (int i = 0; i < S.nsub; ++i)
    for (int k = 0; k < S.K[i]; ++k, ++q) {
      if (!L.psym[q])
        GDSW_CUDA(cudaMemcpyAsync(packed + L.pS[q], fac + S.fS[i][k], sizeof(T) * S.s[i][k] * S.ldS[i][k],
                                  cudaMemcpyDeviceToDevice, s));
      if (k > 0)
        GDSW_CUDA(cudaMemcpyAsync(packed + L.pG[q], fac + S.fG[i][k], sizeof(T) * S.m[i][k] * S.ldG[i][k],
                                  cudaMemcpyDeviceToDevice, s));
    }
  const int cprec = sizeof(T) == 8 ? GDSW_FP64 : GDSW_FP32;
  if (prec == GDSW_BF16) {
    L.fac = c->arena.alloc<__nv_bfloat16>(std::max<int64_t>(off, 1));
    convert(packed, cprec, L.fac, GDSW_BF16, off, s);
  } else {
    L.fac = c->arena.alloc<T>(std::max<int64_t>(off, 1));
    GDSW_CUDA(cudaMemcpyAsync(L.fac, packed, sizeof(T) * off, cudaMemcpyDeviceToDevice, s));
  }
  GDSW_CUDA(cudaStreamSynchronize(s));
  tmp.release(packed);
}

// ------------------------------------------------------------------ level 1 numeric set-up
template <typename T>
static void level1_locals(gdsw_ctx* c, double& minpiv) {
  const SlabSet& S = c->lh[0].loc;
  LevelDev& L = c->ld[0];
  cudaStream_t s = c->stream;
  MatView A = matview(c);
  DevArena tmp(s);
  T* fac = tmp.alloc<T>(S.nfac);
  GDSW_CUDA(cudaMemsetAsync(fac, 0, S.nfac * sizeof(T), s));
  std::vector<int32_t> owner;
  SlabView SV = upload_slabview(tmp, S, s, &owner);
  int* err = tmp.alloc<int>(1);
  GDSW_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  // batches of parts with a private global-to-local map each
  int64_t per_map = c->mesh.n;
  int batch = int(std::max<int64_t>(1, std::min<int64_t>(S.nsub, (int64_t(2) << 30) / (4 * per_map))));
  int32_t* map = tmp.alloc<int32_t>(size_t(batch) * per_map);
  GDSW_CUDA(cudaMemsetAsync(map, 0xff, size_t(batch) * per_map * 4, s));
  for (int i0 = 0; i0 < S.nsub; i0 += batch) {
    int i1 = std::min(S.nsub, i0 + batch);
    extract_slabs<T>(A, SV, S.voff[i0], S.voff[i1], i0, 1, map, fac, err, s);
  }
  int herr = 0;
  GDSW_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  GDSW_CUDA(cudaStreamSynchronize(s));
  GDSW_CHECK(herr == 0, GDSW_ERR_INVALID_ARG, "slab ordering leaves a coupling outside the block tridiagonal");
  tmp.release(map);
  factor_slabs<T>(S, fac, minpiv, s);
  store_factors<T>(c, S, fac, L, c->opt.precision[0], tmp);
  tmp.free_all();
}

template <typename T>
static void level1_coarse(gdsw_ctx* c, double* A0, double& minpiv) {
  const LevelHost& H = c->lh[0];
  const SlabSet& S = H.inter;
  const CoarseSpace& C = H.cs;
  cudaStream_t s = c->stream;
  MatView A = matview(c);
  DevArena tmp(s);
  try {
    T* fac = tmp.alloc<T>(S.nfac);
    GDSW_CUDA(cudaMemsetAsync(fac, 0, S.nfac * sizeof(T), s));
    std::vector<int32_t> owner;
    SlabView SV = upload_slabview(tmp, S, s, &owner);
    int* err = tmp.alloc<int>(1);
    GDSW_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    int32_t* map = tmp.alloc<int32_t>(c->mesh.n);
    GDSW_CUDA(cudaMemsetAsync(map, 0xff, c->mesh.n * 4, s));
    extract_slabs<T>(A, SV, 0, S.nvec, 0, 0, map, fac, err, s);
    factor_slabs<T>(S, fac, minpiv, s);
    // right-hand sides Tneg = -A_IGamma Phi_Gamma
    CSBuild B = cs_layout(C);
    // Phi_Gamma entries by dof: gamma_ptr[g] .. gamma_ptr[g + 1] index gcol / gval (gdofs ascending)
    std::vector<int32_t> gamma_ptr(c->mesh.n + 1, 0), ilocal(c->mesh.n, -1);
    for (int32_t g : C.gdofs) ++gamma_ptr[g + 1];
    for (int64_t g = 0; g < c->mesh.n; ++g) gamma_ptr[g + 1] += gamma_ptr[g];
    for (int64_t p = 0; p < S.nvec; ++p) ilocal[S.gdof[p]] = int32_t(p);
    int32_t* d_gc = tmp.upload(gamma_ptr, s);
    int32_t* d_gcol = tmp.upload(C.gcol, s);
    double* d_gval = tmp.upload(C.gval, s);
    int32_t* d_il = tmp.upload(ilocal, s);
    int32_t* d_cols = tmp.upload(C.cols, s);
    int64_t* d_coff = tmp.upload(C.coff, s);
    int64_t* d_toff = tmp.upload(B.toff, s);
    int32_t* d_ldt = tmp.upload(B.ldt, s);
    double* Tn = tmp.alloc<double>(B.ttot);
    GDSW_CUDA(cudaMemsetAsync(Tn, 0, B.ttot * 8, s));
    launch_tneg(A, SV, d_gc, d_gcol, d_gval, d_cols, d_coff, d_toff, d_ldt, Tn, err, s);
    int herr = 0;
    GDSW_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    GDSW_CUDA(cudaStreamSynchronize(s));
    GDSW_CHECK(herr == 0, GDSW_ERR_INVALID_ARG, "interior coupling outside the part's coarse columns");
    // X = A_II^{-1} Tneg  (= Phi_I)
    T* R = tmp.alloc<T>(B.ttot);
    T* W = tmp.alloc<T>(B.ttot);
    GDSW_CUDA(cudaMemsetAsync(W, 0, B.ttot * sizeof(T), s));
    if (sizeof(T) == 8)
      GDSW_CUDA(cudaMemcpyAsync(R, Tn, B.ttot * 8, cudaMemcpyDeviceToDevice, s));
    else
      convert(Tn, GDSW_FP64, R, GDSW_FP32, B.ttot, s);
    sweep_multi<T>(S, fac, R, W, B.toff, B.ldt, B.nc, s);
    tmp.release(R);
    tmp.release(fac);
    double* X = nullptr;
    if (sizeof(T) == 8) {
      X = reinterpret_cast<double*>(W);
    } else {
      X = tmp.alloc<double>(B.ttot);
      convert(W, GDSW_FP32, X, GDSW_FP64, B.ttot, s);
    }
    // Galerkin product A_0 = Phi^T A Phi = sum_i [X_i^T (A_II X_i - Tn_i) - Tn_i^T X_i] + Phi_G^T A_GG Phi_G
    double* Y = tmp.alloc<double>(B.ttot);
    launch_yint(A, SV, d_il, d_coff, d_toff, d_ldt, X, Tn, Y, s);
    std::vector<int64_t> zoff(C.nparts + 1, 0);
    for (int J = 0; J < C.nparts; ++J) zoff[J + 1] = zoff[J] + int64_t(B.nc[J]) * B.ldt[J];
    double* Z = tmp.alloc<double>(std::max<int64_t>(zoff[C.nparts], 1));
    GDSW_CUDA(cudaMemsetAsync(Z, 0, std::max<int64_t>(zoff[C.nparts], 1) * 8, s));
    std::vector<GemmTaskP> g1, g2;
    for (int J = 0; J < C.nparts; ++J) {
      int nc = B.nc[J];
      int nI = int(C.ioff[J + 1] - C.ioff[J]);
      if (nc == 0 || nI == 0) continue;
      g1.push_back({X + B.toff[J], Y + B.toff[J], Z + zoff[J], nc, nc, nI, B.ldt[J], B.ldt[J], B.ldt[J], 1, 0, 1.0, 0.0});
      g2.push_back({Tn + B.toff[J], X + B.toff[J], Z + zoff[J], nc, nc, nI, B.ldt[J], B.ldt[J], B.ldt[J], 1, 0, -1.0, 1.0});
    }
    run_gemm<double>(tmp, g1, s);
    run_gemm<double>(tmp, g2, s);
    const int64_t n0 = C.n0;
    {
      std::vector<std::pair<int64_t, int64_t>> kv;
      for (int J = 0; J < C.nparts; ++J) {
        int nc = B.nc[J];
        const int32_t* cj = C.cols.data() + C.coff[J];
        for (int a = 0; a < nc; ++a)
          for (int b = 0; b < nc; ++b) kv.push_back({int64_t(cj[a]) * n0 + cj[b], zoff[J] + int64_t(a) * B.ldt[J] + b});
      }
      SegList L = make_segments(kv);
      run_segments(c, L, Z, A0, tmp);
    }
    {
      // interface-interface couplings: positions into the value array
      const MeshHost& M = c->mesh;
      // (Phi_G^T A_GG Phi_G)_{kl} = sum over entries (a, k, w_a) and (b, l, w_b) of w_a w_b A_ab
      std::vector<std::tuple<int64_t, int64_t, double>> kvw;
      const int64_t bt0 = 9 * c->nnzb, b0 = bt0 + 3 * c->nbt;
      for (int k = 0; k < C.n0; ++k) {
        std::vector<std::tuple<int, int64_t, double>> row;
        auto add = [&](int64_t b, int64_t pos, double wa) {
          for (int32_t e = gamma_ptr[b]; e < gamma_ptr[b + 1]; ++e) row.emplace_back(C.gcol[e], pos, wa * C.gval[e]);
        };
        for (int32_t e = C.rg_ptr[k]; e < C.rg_ptr[k + 1]; ++e) {
          int64_t a = C.rg_dof[e];
          const double wa = C.rg_val[e];
          if (a < M.nu) {
            int64_t I = a / 3;
            int cc = int(a - 3 * I);
            for (int32_t blk = M.a_ptr[I]; blk < M.a_ptr[I + 1]; ++blk)
              for (int d = 0; d < 3; ++d) add(3 * int64_t(M.a_col[blk]) + d, int64_t(blk) * 9 + cc * 3 + d, wa);
            for (int32_t q = M.bt_ptr[I]; q < M.bt_ptr[I + 1]; ++q) add(M.nu + M.bt_col[q], bt0 + int64_t(q) * 3 + cc, wa);
          } else {
            int64_t P = a - M.nu;
            for (int32_t q = M.b_ptr[P]; q < M.b_ptr[P + 1]; ++q)
              for (int d = 0; d < 3; ++d) add(3 * int64_t(M.b_col[q]) + d, b0 + int64_t(q) * 3 + d, wa);
          }
        }
        std::stable_sort(row.begin(), row.end(),
                         [](const auto& x, const auto& y) { return std::get<0>(x) < std::get<0>(y); });
        for (auto& pr : row) kvw.emplace_back(int64_t(k) * n0 + std::get<0>(pr), std::get<1>(pr), std::get<2>(pr));
      }
      SegList L = make_segments_w(kvw);
      run_segments(c, L, c->d_val, A0, tmp);
    }
    // store Phi_I^T in the storage precision
    std::vector<int32_t> phild;
    std::vector<int64_t> phioff = phi_offsets(C, phild);
    int64_t* d_phioff = tmp.upload(phioff, s);
    int32_t* d_phild = tmp.upload(phild, s);
    int32_t* d_por = tmp.upload(B.part_of_irow, s);
    int64_t* d_ioff = tmp.upload(C.ioff, s);
    LevelDev& L = c->ld[0];
    if (L.phi_prec == GDSW_FP64)
      store_phiT<double>(X, d_toff, d_ldt, d_por, d_ioff, S.nvec, d_coff, d_phioff, d_phild,
                         static_cast<double*>(L.phiT), nullptr, nullptr, nullptr, 0, s);
    else
      store_phiT<float>(X, d_toff, d_ldt, d_por, d_ioff, S.nvec, d_coff, d_phioff, d_phild,
                        static_cast<float*>(L.phiT), nullptr, nullptr, nullptr, 0, s);
    GDSW_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    tmp.free_all();
    throw;
  }
  tmp.free_all();
}

// ------------------------------------------------------------------ coarse levels (dense operators)
template <typename T>
static void coarse_locals(gdsw_ctx* c, int l, double& minpiv) {
  const SlabSet& S = c->lh[l].loc;
  LevelDev& L = c->ld[l];
  cudaStream_t s = c->stream;
  DevArena tmp(s);
  T* fac = tmp.alloc<T>(S.nfac);
  GDSW_CUDA(cudaMemsetAsync(fac, 0, S.nfac * sizeof(T), s));
  std::vector<int64_t> oo(S.nsub);
  std::vector<int32_t> ol(S.nsub), por;
  for (int i = 0; i < S.nsub; ++i) {
    oo[i] = S.K[i] ? S.fS[i][0] : 0;
    ol[i] = S.K[i] ? S.ldS[i][0] : 8;
    for (int64_t r = S.voff[i]; r < S.voff[i + 1]; ++r) por.push_back(i);
  }
  int32_t* d_dofs = tmp.upload(S.gdof, s);
  int64_t* d_voff = tmp.upload(S.voff, s);
  int32_t* d_por = tmp.upload(por, s);
  int64_t* d_oo = tmp.upload(oo, s);
  int32_t* d_ol = tmp.upload(ol, s);
  gather_dense<T>(L.A, L.n, d_dofs, d_voff, d_por, S.nvec, d_oo, d_ol, fac, s);
  std::vector<InvTaskP> inv;
  for (int i = 0; i < S.nsub; ++i)
    if (S.K[i]) inv.push_back({fac + S.fS[i][0], S.s[i][0], S.ldS[i][0], 0});
  std::vector<double> mp;
  run_inverse<T>(tmp, inv, mp, s);
  minpiv = 1e300;
  for (double v : mp) minpiv = std::min(minpiv, v);
  store_factors<T>(c, S, fac, L, c->opt.precision[l], tmp);
  tmp.free_all();
}

// coarse basis of a coarse level and the next coarse operator A0n = Phi^T A Phi (FP64)
static void coarse_basis(gdsw_ctx* c, int l, double* A0n, double& minpiv) {
  const LevelHost& H = c->lh[l];
  const SlabSet& S = H.inter;
  const CoarseSpace& C = H.cs;
  LevelDev& L = c->ld[l];
  cudaStream_t s = c->stream;
  const int64_t n = L.n, n0 = C.n0;
  DevArena tmp(s);
  try {
    double* fac = tmp.alloc<double>(S.nfac);
    GDSW_CUDA(cudaMemsetAsync(fac, 0, S.nfac * 8, s));
    std::vector<int64_t> oo(S.nsub);
    std::vector<int32_t> ol(S.nsub);
    for (int i = 0; i < S.nsub; ++i) {
      oo[i] = S.K[i] ? S.fS[i][0] : 0;
      ol[i] = S.K[i] ? S.ldS[i][0] : 8;
    }
    CSBuild B = cs_layout(C);
    int32_t* d_idofs = tmp.upload(C.idofs, s);
    int64_t* d_ioff = tmp.upload(C.ioff, s);
    int32_t* d_por = tmp.upload(B.part_of_irow, s);
    int64_t* d_oo = tmp.upload(oo, s);
    int32_t* d_ol = tmp.upload(ol, s);
    gather_dense<double>(L.A, n, d_idofs, d_ioff, d_por, S.nvec, d_oo, d_ol, fac, s);
    std::vector<InvTaskP> inv;
    for (int i = 0; i < S.nsub; ++i)
      if (S.K[i]) inv.push_back({fac + S.fS[i][0], S.s[i][0], S.ldS[i][0], 0});
    std::vector<double> mp;
    run_inverse<double>(tmp, inv, mp, s);
    minpiv = 1e300;
    for (double v : mp) minpiv = std::min(minpiv, v);
    int32_t* d_gd = tmp.upload(C.gdofs, s);
    int32_t* d_gc = tmp.upload(C.gcol, s);
    int32_t* d_cols = tmp.upload(C.cols, s);
    int64_t* d_coff = tmp.upload(C.coff, s);
    int64_t* d_toff = tmp.upload(B.toff, s);
    int32_t* d_ldt = tmp.upload(B.ldt, s);
    double* Tn = tmp.alloc<double>(std::max<int64_t>(B.ttot, 1));
    GDSW_CUDA(cudaMemsetAsync(Tn, 0, std::max<int64_t>(B.ttot, 1) * 8, s));
    coarse_tneg(L.A, n, d_idofs, d_ioff, d_por, S.nvec, d_gd, d_gc, int64_t(C.gdofs.size()), d_cols, d_coff, d_toff,
                d_ldt, Tn, s);
    double* X = tmp.alloc<double>(std::max<int64_t>(B.ttot, 1));
    std::vector<GemmTaskP> g;
    for (int J = 0; J < C.nparts; ++J) {
      int nI = int(C.ioff[J + 1] - C.ioff[J]);
      if (nI == 0 || B.nc[J] == 0) continue;
      g.push_back({fac + S.fS[J][0], Tn + B.toff[J], X + B.toff[J], nI, B.nc[J], nI, S.ldS[J][0], B.ldt[J], B.ldt[J],
                   0, 0, 1.0, 0.0});
    }
    run_gemm<double>(tmp, g, s);
    double* dense = tmp.alloc<double>(n * n0);
    GDSW_CUDA(cudaMemsetAsync(dense, 0, n * n0 * 8, s));
    std::vector<int32_t> phild;
    std::vector<int64_t> phioff = phi_offsets(C, phild);
    int64_t* d_phioff = tmp.upload(phioff, s);
    int32_t* d_phild = tmp.upload(phild, s);
    if (L.phi_prec == GDSW_FP64)
      store_phiT<double>(X, d_toff, d_ldt, d_por, d_ioff, S.nvec, d_coff, d_phioff, d_phild,
                         static_cast<double*>(L.phiT), d_idofs, d_cols, dense, n0, s);
    else
      store_phiT<float>(X, d_toff, d_ldt, d_por, d_ioff, S.nvec, d_coff, d_phioff, d_phild, static_cast<float*>(L.phiT),
                        d_idofs, d_cols, dense, n0, s);
    dense_gamma(d_gd, d_gc, int64_t(C.gdofs.size()), dense, n0, s);
    double* T1 = tmp.alloc<double>(n * n0);
    run_gemm<double>(tmp, {{L.A, dense, T1, int(n), int(n0), int(n), int(n), int(n0), int(n0), 0, 0, 1.0, 0.0}}, s);
    run_gemm<double>(tmp, {{dense, T1, A0n, int(n0), int(n0), int(n), int(n0), int(n0), int(n0), 1, 0, 1.0, 0.0}}, s);
    GDSW_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    tmp.free_all();
    throw;
  }
  tmp.free_all();
}

// ------------------------------------------------------------------ apply
static void local_solve(gdsw_ctx* c, int l, const double* r, double* z, cudaStream_t s) {
  LevelDev& L = c->ld[l];
  const LevelHost& H = c->lh[l];
  const int64_t nv = L.nvec;
  double gbytes = 0;
  {
    // level-1 groups carry only level-1 work; every coarser level's work is the "coarse" group
    ProfScope ps(c, l == 0 ? GDSW_K_GATHER : GDSW_K_COARSE, double(nv) * (4 + 8 + (L.prec == GDSW_FP64 ? 8 : 4)), s);
    if (L.prec == GDSW_FP64)
      launch_gather<double>(r, L.gdof, static_cast<double*>(L.vec), nv, s);
    else
      launch_gather<float>(r, L.gdof, static_cast<float*>(L.vec), nv, s);
  }
  // block-LDL^T sweeps: forward launches (S_k^{-1} y_k and the G_{k+1} update), then backward
  // launches (G_{k+1}^T), every one a ragged batched GEMV over all parts of the level
  const int group = l == 0 ? GDSW_K_LOCAL : GDSW_K_COARSE;
  auto sweep = [&](const GemvPlan& P, int k, int ld) {
    if (L.prec == GDSW_FP64) {
      double* v = static_cast<double*>(L.vec);
      launch_gemv<double, double>(static_cast<const double*>(L.fac), v, v, v, P, k, ld, s);
    } else if (L.prec == GDSW_FP32) {
      float* v = static_cast<float*>(L.vec);
      launch_gemv<float, float>(static_cast<const float*>(L.fac), v, v, v, P, k, ld, s);
    } else {
      float* v = static_cast<float*>(L.vec);
      launch_gemv<__nv_bfloat16, float>(static_cast<const __nv_bfloat16*>(L.fac), v, v, v, P, k, ld, s);
    }
  };
  if (L.persistent && L.sweep.nitems > 0) {
    // the whole forward / reduction / backward sequence as one persistent launch
    double bytes = L.red_bytes;
    for (double b : L.fwd_bytes) bytes += b;
    for (double b : L.bwd_bytes) bytes += b;
    ProfScope ps(c, group, bytes, s);
    if (L.prec == GDSW_FP64)
      launch_sweep<double, double>(static_cast<const double*>(L.fac), static_cast<double*>(L.vec), L.sweep,
                                   c->d_sweep_flag, L.sym_T, s);
    else if (L.prec == GDSW_FP32)
      launch_sweep<float, float>(static_cast<const float*>(L.fac), static_cast<float*>(L.vec), L.sweep,
                                 c->d_sweep_flag, L.sym_T, s);
    else
      launch_sweep<__nv_bfloat16, float>(static_cast<const __nv_bfloat16*>(L.fac), static_cast<float*>(L.vec),
                                         L.sweep, c->d_sweep_flag, L.sym_T, s);
  } else {
  // the chained launches are timed as one unit: events between them would break the chain
  double bytes = L.red_bytes;
  for (double b : L.fwd_bytes) bytes += b;
  for (double b : L.bwd_bytes) bytes += b;
  ProfScope ps(c, group, bytes, s);
  for (int k = 0; k < L.fwd.nlaunch(); ++k) sweep(L.fwd, k, L.fwd_ld[k]);
  if (L.red.launch_tile_off.size() == 2 && L.red.launch_tile_off[1] > 0) {
    // w_k = S_k^{-1} y_k of the packed symmetric blocks: sum of the partial products
    if (L.prec == GDSW_FP64)
      launch_sym_reduce<double>(static_cast<const double*>(L.vec), static_cast<double*>(L.vec), L.red, L.sym_T, s);
    else
      launch_sym_reduce<float>(static_cast<const float*>(L.vec), static_cast<float*>(L.vec), L.red, L.sym_T, s);
  }
  for (int k = 0; k < L.bwd.nlaunch(); ++k) sweep(L.bwd, k, L.bwd_ld[k]);
  }
  {
    ProfScope ps(c, l == 0 ? GDSW_K_SCATTER : GDSW_K_COARSE,
                 double(nv) * (4 + 8 + (L.prec == GDSW_FP64 ? 8 : 4)) + 8.0 * L.n, s);
    if (L.prec == GDSW_FP64)
      launch_scatter<double>(static_cast<const double*>(L.vec) + nv, L.sc_ptr, L.sc_pos, L.sc_w, z, L.n, 0, s);
    else
      launch_scatter<float>(static_cast<const float*>(L.vec) + nv, L.sc_ptr, L.sc_pos, L.sc_w, z, L.n, 0, s);
  }
  (void)H;
  (void)gbytes;
}

// algorithmic bytes of one preconditioner apply (all levels), for the apply GB/s figure
static double apply_bytes(const gdsw_ctx* c) {
  double b = 0;
  for (size_t l = 0; l < c->ld.size(); ++l) {
    const LevelDev& L = c->ld[l];
    const double vs = L.prec == GDSW_FP64 ? 8 : 4;
    b += double(L.nvec) * (4 + 8 + vs) * 2 + 8.0 * L.n;                // gather + scatter
    for (double x : L.fwd_bytes) b += x;
    for (double x : L.bwd_bytes) b += x;
    b += L.red_bytes;
    if (L.n0) b += 2 * (L.phi_bytes + 16.0 * L.nidofs + 16.0 * L.ngamma);  // Phi^T and Phi
  }
  b += 8.0 * double(c->n_coarsest) * c->ld_coarsest;
  return b;
}

static void restrict_level(gdsw_ctx* c, int l, const double* r, double* r0, cudaStream_t s) {
  LevelDev& L = c->ld[l];
  if (L.n0 == 0) return;
  ProfScope ps(c, l == 0 ? GDSW_K_RESTRICT : GDSW_K_COARSE, double(L.phi_bytes) + 16.0 * L.nidofs, s);
  launch_restrict(L, r, r0, s);
}

static void coarsest_solve(gdsw_ctx* c, const double* r0, double* x0, cudaStream_t s) {
  ProfScope ps(c, GDSW_K_COARSE, 8.0 * double(c->n_coarsest) * c->ld_coarsest, s);
  launch_gemv<double, double>(c->d_coarsest_inv, r0, x0, nullptr, c->coarsest_plan, 0, c->ld_coarsest, s);
}

static void apply_level(gdsw_ctx* c, int l, const double* r, double* z, cudaStream_t s) {
  LevelDev& L = c->ld[l];
  const int nlev = int(c->ld.size());
  const bool coarse = L.n0 > 0;
  const bool fork = coarse && l == 0 && c->stream2 != nullptr;
  cudaStream_t sc = fork ? c->stream2 : s;
  if (fork) {
    GDSW_CUDA(cudaEventRecord(c->ev_fork, s));
    GDSW_CUDA(cudaStreamWaitEvent(sc, c->ev_fork, 0));
  }
  if (coarse) {
    restrict_level(c, l, r, L.r0, sc);
    if (l + 1 < nlev)
      apply_level(c, l + 1, L.r0, L.x0, sc);
    else
      coarsest_solve(c, L.r0, L.x0, sc);
  }
  local_solve(c, l, r, z, s);
  if (fork) {
    GDSW_CUDA(cudaEventRecord(c->ev_join, sc));
    GDSW_CUDA(cudaStreamWaitEvent(s, c->ev_join, 0));
  }
  if (coarse) {
    {  // interior part z_I += Phi_I x0 (k_prolong): the basis once plus the read-modify-write of z_I
      ProfScope ps(c, l == 0 ? GDSW_K_PROLONG : GDSW_K_COARSE, double(L.phi_bytes) + 16.0 * L.nidofs, s);
      launch_prolong(L, L.x0, z, s);
    }
    {  // interface part z_G += Phi_G x0: per entry column and value, per dof its index and z
      ProfScope ps(c, l == 0 ? GDSW_K_OTHER : GDSW_K_COARSE, 12.0 * L.ngamma + 24.0 * L.ngu, s);
      launch_axpy_gamma(L.gu_dof, L.gu_ptr, L.gcol, L.gval, L.ngu, L.x0, z, s);
    }
  }
}

static void apply_precond_impl(gdsw_ctx* c, const double* r, double* z, cudaStream_t s) {
  apply_level(c, 0, r, z, s);
}

void apply_precond(gdsw_ctx* c, const double* r, double* z, cudaStream_t s) {
  if (c->ext_precond) {  // a preconditioner attached from outside (the multigrid V-cycle)
    c->ext_precond(c->ext_data, r, z, s);
    return;
  }
  GDSW_CHECK(!c->ld.empty(), GDSW_ERR_INVALID_ARG, "operator-only context has no preconditioner");
  if (c->prof.enabled) {
    c->prof_gate = (c->apply_count % c->prof_stride) == 0;
    ++c->apply_count;
  }
  if (c->apply_graph && !(c->prof.enabled && c->prof_gate)) {
    GDSW_CUDA(cudaMemcpyAsync(c->d_graph_r, r, sizeof(double) * c->mesh.n, cudaMemcpyDeviceToDevice, s));
    GDSW_CUDA(cudaGraphLaunch(c->apply_graph, s));
    GDSW_CUDA(cudaMemcpyAsync(z, c->d_graph_z, sizeof(double) * c->mesh.n, cudaMemcpyDeviceToDevice, s));
    return;
  }
  ProfScope ps(c, GDSW_K_APPLY, c->apply_bytes, s);
  apply_level(c, 0, r, z, s);
}

static void capture_graph(gdsw_ctx* c) {
  c->d_graph_r = c->arena.alloc<double>(c->mesh.n);
  c->d_graph_z = c->arena.alloc<double>(c->mesh.n);
  GDSW_CUDA(cudaMemsetAsync(c->d_graph_r, 0, 8 * c->mesh.n, c->stream));
  GDSW_CUDA(cudaStreamSynchronize(c->stream));
  // capture on a private stream (the caller's stream may be the legacy default stream)
  cudaStream_t cs;
  GDSW_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g;
  GDSW_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  try {
    c->capturing = true;
    apply_level(c, 0, c->d_graph_r, c->d_graph_z, cs);
    c->capturing = false;
  } catch (...) {
    c->capturing = false;
    cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    throw;
  }
  GDSW_CUDA(cudaStreamEndCapture(cs, &g));
  GDSW_CUDA(cudaGraphInstantiate(&c->apply_graph, g, 0));
  GDSW_CUDA(cudaGraphDestroy(g));
  GDSW_CUDA(cudaStreamDestroy(cs));
}

// ------------------------------------------------------------------ set-up driver
void setup_impl(gdsw_ctx* c, const gdsw_mesh* mesh, const gdsw_viscosity* visc, const gdsw_partition* part,
                const gdsw_levels* lv, const gdsw_options* opt) {
  GDSW_CHECK(mesh && visc && part && lv && opt, GDSW_ERR_INVALID_ARG, "null argument");
  GDSW_CHECK(mesh->nx > 0 && mesh->ny > 0 && mesh->nz > 0 && mesh->h > 0, GDSW_ERR_INVALID_ARG, "bad mesh size");
  GDSW_CHECK(mesh->mask && mesh->tags && mesh->g && part->elem_part, GDSW_ERR_INVALID_ARG, "null mesh array");
  GDSW_CHECK(lv->levels >= 1 && lv->levels <= 4, GDSW_ERR_INVALID_ARG, "levels must be 1 (operator only), 2, 3 or 4");
  GDSW_CHECK(part->n_groups == std::max(lv->levels - 2, 0), GDSW_ERR_INVALID_ARG, "need levels-2 grouping arrays");
  GDSW_CHECK(lv->overlap >= 1 && lv->overlap <= 4, GDSW_ERR_INVALID_ARG, "overlap must be 1..4");
  GDSW_CHECK(opt->slab_elems >= 0, GDSW_ERR_INVALID_ARG, "slab_elems must be >= 0");
  for (int l = 0; l < lv->levels - 1; ++l)
    GDSW_CHECK(opt->precision[l] >= GDSW_FP64 && opt->precision[l] <= GDSW_BF16, GDSW_ERR_INVALID_ARG, "bad precision");
  GDSW_CHECK(opt->phi_precision == GDSW_FP64 || opt->phi_precision == GDSW_FP32, GDSW_ERR_INVALID_ARG,
             "phi precision must be FP64 or FP32");
  GDSW_CHECK(visc->form == GDSW_FORM_GRADIENT || visc->form == GDSW_FORM_SYMMETRIC, GDSW_ERR_INVALID_ARG, "bad form");
  c->opt = *opt;
  if (c->opt.restart <= 0) c->opt.restart = 100;
  if (c->opt.max_it <= 0) c->opt.max_it = 1000;
  c->L = lv->levels;
  double t0 = now_ms();
  const int nlev = c->L - 1;
  if (!c->host_ready) {
    // ---- host symbolic set-up (shared by gdsw_analyze, gdsw_setup and the server's admission)
    build_mesh(c->mesh, mesh);
    c->lh.assign(nlev, LevelHost());
    GDSW_CHECK(lv->rotations == 0 || lv->levels == 2, GDSW_ERR_INVALID_ARG, "rotation modes need two levels");
    if (nlev > 0) build_level1(c, part, lv->overlap, opt->slab_elems, lv->rotations);
    for (int l = 1; l < nlev; ++l) {
      GDSW_CHECK(part->groups[l - 1] != nullptr, GDSW_ERR_INVALID_ARG, "null grouping array");
      build_coarse_level(c, l, part->groups[l - 1], part->group_len[l - 1]);
    }
    c->setup_ms[0] = now_ms() - t0;
    // device memory the full set-up would hold (factors, bases, operator, Krylov space)
    const MeshHost& M = c->mesh;
    double b = 8.0 * (9.0 * M.a_col.size() + 3.0 * M.bt_col.size() + 3.0 * M.b_col.size());
    b += 4.0 * (M.a_col.size() + M.bt_col.size() + M.b_col.size() + 4.0 * M.n) + 8.0 * 27 * M.fluid.size();
    b += 4.0 * (M.asm_uoff.size() + M.asm_unit.size() + M.asm_cta.size());
    b += 80.0 * M.sell_acol.size() + 32.0 * M.sell_bcol.size() + 4.0 * M.sell_row.size();
    for (int l = 0; l < nlev; ++l) {
      const LevelHost& H = c->lh[l];
      b += double(H.loc.nfac) * elem_size(opt->precision[l]) + 16.0 * H.loc.nvec + 16.0 * H.loc.nvec;
      for (int J = 0; J < H.cs.nparts; ++J)  // Phi_I^T blocks
        b += double(H.cs.ioff[J + 1] - H.cs.ioff[J]) * double(H.cs.coff[J + 1] - H.cs.coff[J]) *
             elem_size(l == 0 ? opt->phi_precision : GDSW_FP64);
    }
    b += 8.0 * (2.0 * c->opt.restart + 2.0) * M.n;
    // the factorisation works in a temporary copy of the level-1 factors and interiors
    if (nlev > 0) b += double(c->lh[0].loc.nfac) * (opt->precision[0] == GDSW_FP64 ? 8 : 4);
    c->est_device_bytes = int64_t(b);
    c->host_ready = true;
  }
  if (c->host_only) return;
  // NULL selects the legacy default stream, so calls order with other default-stream work
  c->stream = static_cast<cudaStream_t>(opt->stream);
  GDSW_CUDA(cudaGetDevice(&c->device));
  GDSW_CUDA(cudaStreamCreateWithFlags(&c->stream2, cudaStreamNonBlocking));
  GDSW_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  GDSW_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  cudaStream_t s = c->stream;
  c->arena.stream = s;  // context memory is allocated and freed in the order of its stream
  c->arena.ordered = true;
  set_gemv_smem_limits();
  set_prolong_smem_limits();
  c->ld.assign(nlev, LevelDev());
  double t1 = now_ms();
  // ---- device mesh and operator
  MeshHost& M = c->mesh;
  c->form = visc->form;
  c->nu0 = visc->nu0;
  c->nu_inf = visc->nu_inf;
  c->lam = visc->lambda;
  c->ncar = visc->n;
  c->has_uk = visc->uk != nullptr;
  upload_tables(c, s);
  c->d_mask = c->arena.upload(M.mask, s);
  c->d_fluid = c->arena.upload(M.fluid, s);
  c->d_felem = c->arena.upload(M.felem, s);
  c->d_vnode = c->arena.upload(M.vnode, s);
  c->d_pnode = c->arena.upload(M.pnode, s);
  c->d_a_ptr = c->arena.upload(M.a_ptr, s);
  c->d_a_col = c->arena.upload(M.a_col, s);
  c->d_a_diag = c->arena.upload(M.a_diag, s);
  c->d_a_tpos = c->arena.upload(M.a_tpos, s);
  c->d_asm_cta = c->arena.upload(M.asm_cta, s);
  c->d_asm_uoff = c->arena.upload(M.asm_uoff, s);
  c->d_asm_unit = c->arena.upload(M.asm_unit, s);
  c->n_sell_slices = int64_t(M.sell_aoff.size()) - 1;
  c->d_sell_row = c->arena.upload(M.sell_row, s);
  c->d_sell_aoff = c->arena.upload(M.sell_aoff, s);
  c->d_sell_boff = c->arena.upload(M.sell_boff, s);
  c->d_sell_acol = c->arena.upload(M.sell_acol, s);
  c->d_sell_asrc = c->arena.upload(M.sell_asrc, s);
  c->d_sell_bcol = c->arena.upload(M.sell_bcol, s);
  c->d_sell_bsrc = c->arena.upload(M.sell_bsrc, s);
  c->d_sell_aval = c->arena.alloc<double>(9 * M.sell_acol.size());
  c->d_sell_btval = c->arena.alloc<double>(3 * M.sell_bcol.size());
  c->d_bt_ptr = c->arena.upload(M.bt_ptr, s);
  c->d_bt_col = c->arena.upload(M.bt_col, s);
  c->d_b_ptr = c->arena.upload(M.b_ptr, s);
  c->d_b_col = c->arena.upload(M.b_col, s);
  c->d_bt2b = c->arena.upload(M.bt2b, s);
  c->d_ad_ptr = c->arena.upload(M.ad_ptr, s);
  c->d_ad_col = c->arena.upload(M.ad_col, s);
  c->d_bd_ptr = c->arena.upload(M.bd_ptr, s);
  c->d_bd_col = c->arena.upload(M.bd_col, s);
  {
    std::vector<int32_t> rows;
    for (int64_t r = 0; r < M.nv; ++r)
      if (M.ad_ptr[r + 1] > M.ad_ptr[r]) rows.push_back(int32_t(r));
    for (int64_t P = 0; P < M.np; ++P)
      if (M.bd_ptr[P + 1] > M.bd_ptr[P]) rows.push_back(int32_t(M.nv + P));
    c->n_lift_rows = int64_t(rows.size());
    c->d_lift_rows = rows.empty() ? nullptr : c->arena.upload(rows, s);
  }
  c->d_sweep_flag = c->arena.alloc<unsigned>(1);
  GDSW_CUDA(cudaMemsetAsync(c->d_sweep_flag, 0, sizeof(unsigned), s));
  c->d_gdir = c->arena.upload(M.g, s);
  c->d_uk = c->arena.alloc<double>(3 * M.nnodes);
  if (visc->uk)
    GDSW_CUDA(cudaMemcpyAsync(c->d_uk, visc->uk, 24 * M.nnodes, cudaMemcpyHostToDevice, s));
  c->d_nu = c->arena.alloc<double>(27 * M.fluid.size());
  c->nnzb = int64_t(M.a_col.size());
  c->nbt = int64_t(M.bt_col.size());
  c->nb = int64_t(M.b_col.size());
  c->d_val = c->arena.alloc<double>(9 * c->nnzb + 3 * c->nbt + 3 * c->nb);
  launch_viscosity(c, s);
  launch_assembly(c, s);
  GDSW_CUDA(cudaStreamSynchronize(s));
  double t2 = now_ms();
  c->setup_ms[1] = t2 - t1;
  if (nlev == 0) {  // operator only: assembly, SpMV and lifting, no Schwarz levels
    c->setup_ms[5] = now_ms() - t0;
    return;
  }
  // ---- level 1
  double minpiv = 0;
  {
    LevelDev& L = c->ld[0];
    L.n = int(M.n);
    L.N = c->lh[0].N;
    const bool f64 = opt->precision[0] == GDSW_FP64;
    if (f64)
      level1_locals<double>(c, minpiv);
    else
      level1_locals<float>(c, minpiv);
    GDSW_CHECK(minpiv > 0 && std::isfinite(minpiv), GDSW_ERR_SINGULAR, "level-1 local factorisation: zero pivot");
    L.minpiv = minpiv;
    const LevelHost& H = c->lh[0];
    L.gdof = c->arena.upload(H.loc.gdof, s);
    L.sc_ptr = c->arena.upload(H.sc_ptr, s);
    L.sc_pos = c->arena.upload(H.sc_pos, s);
    L.sc_w = c->arena.upload(H.sc_w, s);
    build_local_plan(c, H.loc, L);
    // local vectors (y, w) and the symmetric partial sums behind them
    size_t vb = size_t(std::max<int64_t>(2 * H.loc.nvec + L.npart, 1)) * (L.prec == GDSW_FP64 ? 8 : 4);
    L.vec = c->arena.alloc<char>(vb);
    GDSW_CUDA(cudaMemsetAsync(L.vec, 0, vb, s));
    L.local_bytes = double(L.nfac) * elem_size(L.prec) + 2.0 * H.loc.nvec * (L.prec == GDSW_FP64 ? 8 : 4);
  }
  double t3 = now_ms();
  c->setup_ms[2] = t3 - t2;
  // ---- level-1 coarse space and A_0^(2)
  double* A0 = nullptr;
  int64_t n0 = c->lh[0].cs.n0;
  {
    LevelDev& L = c->ld[0];
    upload_coarse_space(c, 0, opt->phi_precision);
    L.phi_bytes = 0;
    if (n0 > 0) {
      A0 = c->arena.alloc<double>(n0 * n0);
      GDSW_CUDA(cudaMemsetAsync(A0, 0, n0 * n0 * 8, s));
      if (opt->phi_precision == GDSW_FP64)
        level1_coarse<double>(c, A0, minpiv);
      else
        level1_coarse<float>(c, A0, minpiv);
      GDSW_CHECK(minpiv > 0 && std::isfinite(minpiv), GDSW_ERR_SINGULAR, "interior factorisation: zero pivot");
      std::vector<int32_t> ld;
      std::vector<int64_t> off = phi_offsets(c->lh[0].cs, ld);
      L.phi_bytes = double(off.back()) * elem_size(opt->phi_precision);
    }
  }
  double t4 = now_ms();
  c->setup_ms[3] = t4 - t3;
  // ---- coarse levels
  for (int l = 1; l < nlev; ++l) {
    LevelDev& L = c->ld[l];
    const LevelHost& H = c->lh[l];
    L.n = H.n;
    L.N = H.N;
    L.A = A0;
    if (opt->precision[l] == GDSW_FP64)
      coarse_locals<double>(c, l, minpiv);
    else
      coarse_locals<float>(c, l, minpiv);
    GDSW_CHECK(minpiv > 0 && std::isfinite(minpiv), GDSW_ERR_SINGULAR, "coarse local factorisation: zero pivot");
    L.minpiv = minpiv;
    L.gdof = c->arena.upload(H.loc.gdof, s);
    L.sc_ptr = c->arena.upload(H.sc_ptr, s);
    L.sc_pos = c->arena.upload(H.sc_pos, s);
    L.sc_w = c->arena.upload(H.sc_w, s);
    build_local_plan(c, H.loc, L);
    size_t vb = size_t(std::max<int64_t>(2 * H.loc.nvec + L.npart, 1)) * (L.prec == GDSW_FP64 ? 8 : 4);
    L.vec = c->arena.alloc<char>(vb);
    GDSW_CUDA(cudaMemsetAsync(L.vec, 0, vb, s));
    L.local_bytes = double(L.nfac) * elem_size(L.prec) + 2.0 * H.loc.nvec * (L.prec == GDSW_FP64 ? 8 : 4);
    upload_coarse_space(c, l, GDSW_FP64);
    int64_t m0 = H.cs.n0;
    double* A0n = nullptr;
    if (m0 > 0) {
      A0n = c->arena.alloc<double>(m0 * m0);
      coarse_basis(c, l, A0n, minpiv);
      GDSW_CHECK(minpiv > 0 && std::isfinite(minpiv), GDSW_ERR_SINGULAR, "coarse interior factorisation: zero pivot");
      std::vector<int32_t> ldv;
      std::vector<int64_t> off = phi_offsets(H.cs, ldv);
      L.phi_bytes = double(off.back()) * 8.0;
    }
    A0 = A0n;
    n0 = m0;
  }
  // ---- coarsest direct solve: explicit FP64 inverse of A_0^(L)
  c->n_coarsest = int(n0);
  c->coarsest_A = A0;
  if (n0 > 0) {
    int ldc = int(pad8(n0));
    c->ld_coarsest = ldc;
    c->d_coarsest_inv = c->arena.alloc<double>(n0 * ldc);
    GDSW_CUDA(cudaMemsetAsync(c->d_coarsest_inv, 0, n0 * ldc * 8, s));
    GDSW_CUDA(cudaMemcpy2DAsync(c->d_coarsest_inv, ldc * 8, A0, n0 * 8, n0 * 8, n0, cudaMemcpyDeviceToDevice, s));
    std::vector<double> hA(n0 * n0);
    GDSW_CUDA(cudaMemcpyAsync(hA.data(), A0, 8 * n0 * n0, cudaMemcpyDeviceToHost, s));
    GDSW_CUDA(cudaStreamSynchronize(s));
    double amax = 0.0;
    for (double v : hA) amax = std::max(amax, std::fabs(v));
    DevArena tmp(s);
    std::vector<double> mp;
    run_inverse<double>(tmp, {{c->d_coarsest_inv, int(n0), ldc, 0}}, mp, s);
    tmp.free_all();
    // direct solve of the smallest level: a pivot below 1e-12 of the largest entry means
    // A_0^(L) is numerically singular (e.g. no Dirichlet data at all)
    GDSW_CHECK(mp[0] > 1e-12 * amax && std::isfinite(mp[0]), GDSW_ERR_SINGULAR, "coarsest operator is singular");
    c->coarsest_minpiv = mp[0];
    std::vector<GemvTask> tasks;
    std::vector<GemvTile> tiles;
    add_task(tasks, tiles, GemvTask{0, 0, 0, -1, int(n0), int(n0), ldc, 1.0f}, c->coarsest_plan.rows_per_tile);
    c->coarsest_plan.launch_task_off = {0, int(tasks.size())};
    c->coarsest_plan.launch_tile_off = {0, int(tiles.size())};
    finish_plan(c->arena, c->coarsest_plan, tasks, tiles, s);
  }
  double t5 = now_ms();
  c->setup_ms[4] = t5 - t4;
  GDSW_CUDA(cudaStreamSynchronize(s));
  autotune_level1(c);
  if (opt->use_graph) capture_graph(c);
  c->apply_bytes = apply_bytes(c);
  c->setup_ms[5] = now_ms() - t0;
}

}  // namespace gdsw

using namespace gdsw;

// ------------------------------------------------------------------ C ABI
#define GDSW_TRY(ctx, body)                                                                  \
  try {                                                                                      \
    body;                                                                                    \
    return GDSW_OK;                                                                          \
  } catch (const gdsw::Error& e) {                                                           \
    if (ctx) (ctx)->err = e.msg;                                                             \
    return e.code;                                                                           \
  } catch (const std::bad_alloc&) {                                                          \
    if (ctx) (ctx)->err = "host allocation failed";                                          \
    return GDSW_ERR_OOM;                                                                     \
  } catch (...) {                                                                            \
    if (ctx) (ctx)->err = "unknown error";                                                   \
    return GDSW_ERR_CUDA;                                                                    \
  }

extern "C" {

int gdsw_setup(const gdsw_mesh* mesh, const gdsw_viscosity* visc, const gdsw_partition* part, const gdsw_levels* lv,
               const gdsw_options* opt, gdsw_ctx** out) {
  if (!out) return GDSW_ERR_INVALID_ARG;
  *out = nullptr;
  gdsw_ctx* c = new (std::nothrow) gdsw_ctx();
  if (!c) return GDSW_ERR_OOM;
  int rc;
  try {
    setup_impl(c, mesh, visc, part, lv, opt);
    rc = GDSW_OK;
  } catch (const gdsw::Error& e) {
    g_setup_error = e.msg;
    rc = e.code;
  } catch (const std::bad_alloc&) {
    g_setup_error = "host allocation failed";
    rc = GDSW_ERR_OOM;
  } catch (...) {
    g_setup_error = "unknown error";
    rc = GDSW_ERR_CUDA;
  }
  if (rc != GDSW_OK) {
    gdsw_destroy(c);
    return rc;
  }
  g_setup_error.clear();
  *out = c;
  return GDSW_OK;
}

int gdsw_analyze(const gdsw_mesh* mesh, const gdsw_viscosity* visc, const gdsw_partition* part,
                 const gdsw_levels* lv, const gdsw_options* opt, gdsw_ctx** out) {
  if (!out) return GDSW_ERR_INVALID_ARG;
  *out = nullptr;
  gdsw_ctx* c = new (std::nothrow) gdsw_ctx();
  if (!c) return GDSW_ERR_OOM;
  c->host_only = true;
  int rc = GDSW_OK;
  try {
    setup_impl(c, mesh, visc, part, lv, opt);
  } catch (const gdsw::Error& e) {
    g_setup_error = e.msg;
    rc = e.code;
  } catch (const std::bad_alloc&) {
    g_setup_error = "host allocation failed";
    rc = GDSW_ERR_OOM;
  }
  if (rc != GDSW_OK) {
    delete c;
    return rc;
  }
  *out = c;
  return GDSW_OK;
}

void gdsw_destroy(gdsw_ctx* c) {
  if (!c) return;
  if (c->host_only) {
    delete c;
    return;
  }
  if (c->stream2) cudaStreamSynchronize(c->stream2);
  cudaStreamSynchronize(c->stream);
  if (c->apply_graph) cudaGraphExecDestroy(c->apply_graph);
  for (auto& p : c->pending) {
    c->ev_pool.push_back(p.a);
    c->ev_pool.push_back(p.b);
  }
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  c->arena.free_all();
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->stream2) cudaStreamDestroy(c->stream2);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* gdsw_last_error(const gdsw_ctx* c) { return c ? c->err.c_str() : g_setup_error.c_str(); }

int gdsw_sizes(const gdsw_ctx* c, gdsw_sizes_info* info) {
  if (!c || !info) return GDSW_ERR_INVALID_ARG;
  gdsw_sizes_info s{};
  s.n = c->mesh.n;
  s.n_u = c->mesh.nu;
  s.n_p = c->mesh.np;
  s.n_elems = int64_t(c->mesh.fluid.size());
  s.n_nodes = c->mesh.nnodes;
  s.levels = c->L;
  for (size_t l = 0; l < c->lh.size() && l < 3; ++l) {
    s.n_coarse[l] = c->lh[l].cs.n0;
    s.n_parts[l] = c->lh[l].N;
    s.local_dofs[l] = c->lh[l].loc.nvec;
    s.factor_entries[l] = c->lh[l].loc.nfac;
    s.max_local[l] = c->lh[l].loc.max_local;
  }
  s.max_slabs = c->lh.empty() ? 0 : c->lh[0].loc.Kmax;
  s.nnzb_A = c->nnzb;
  s.nnz_B = c->nb;
  s.phi_entries = c->lh.empty() ? 0 : int64_t(c->lh[0].cs.idofs.size());
  s.device_bytes = c->host_only ? c->est_device_bytes : int64_t(c->arena.bytes);
  for (int q = 0; q < 6; ++q) s.setup_ms[q] = c->setup_ms[q];
  for (size_t l = 0; l < c->ld.size() && l < 3; ++l) {
    s.tile_rows[l] = c->ld[l].fwd.rows_per_tile;
    s.persistent[l] = c->ld[l].persistent ? 1 : 0;
    s.tuned_ms[l] = c->ld[l].tuned_ms;
  }
  *info = s;
  return GDSW_OK;
}

int gdsw_rhs_lift(gdsw_ctx* c, double* b) {
  if (!c || c->host_only || !b) return GDSW_ERR_INVALID_ARG;
  GDSW_TRY(c, launch_lift(c, b, c->stream));
}

int gdsw_spmv(gdsw_ctx* c, const double* x, double* y) {
  if (!c || c->host_only || !x || !y) return GDSW_ERR_INVALID_ARG;
  GDSW_TRY(c, {
    ProfScope ps(c, GDSW_K_SPMV, c->spmv_bytes(), c->stream);
    launch_spmv(c, x, y, nullptr, c->stream);
  });
}

int gdsw_apply(gdsw_ctx* c, const double* r, double* z) {
  if (!c || c->host_only || !r || !z) return GDSW_ERR_INVALID_ARG;
  GDSW_TRY(c, apply_precond(c, r, z, c->stream));
}

int gdsw_solve(gdsw_ctx* c, const double* b, double* x, gdsw_solve_info* info) {
  if (!c || c->host_only || !b || !x) return GDSW_ERR_INVALID_ARG;
  gdsw_solve_info tmp{};
  if (!info) info = &tmp;
  int rc;
  try {
    fgmres_solve(c, b, x, info);
    rc = info->status;
  } catch (const gdsw::Error& e) {
    c->err = e.msg;
    rc = e.code;
  } catch (...) {
    c->err = "unknown error";
    rc = GDSW_ERR_CUDA;
  }
  return rc;
}

int gdsw_solve_host(gdsw_ctx* c, const double* bh, double* xh, gdsw_solve_info* info) {
  if (!c || c->host_only || !bh || !xh) return GDSW_ERR_INVALID_ARG;
  try {
    if (!c->d_hb) {
      c->d_hb = c->arena.alloc<double>(c->mesh.n);
      c->d_hx = c->arena.alloc<double>(c->mesh.n);
    }
    GDSW_CUDA(cudaMemcpyAsync(c->d_hb, bh, 8 * c->mesh.n, cudaMemcpyHostToDevice, c->stream));
    GDSW_CUDA(cudaMemcpyAsync(c->d_hx, xh, 8 * c->mesh.n, cudaMemcpyHostToDevice, c->stream));
    int rc = gdsw_solve(c, c->d_hb, c->d_hx, info);
    GDSW_CUDA(cudaMemcpyAsync(xh, c->d_hx, 8 * c->mesh.n, cudaMemcpyDeviceToHost, c->stream));
    GDSW_CUDA(cudaStreamSynchronize(c->stream));
    return rc;
  } catch (const gdsw::Error& e) {
    c->err = e.msg;
    return e.code;
  }
}

int gdsw_residual(gdsw_ctx* c, const double* b, const double* x, double* r) {
  if (!c || c->host_only || !b || !x || !r) return GDSW_ERR_INVALID_ARG;
  GDSW_TRY(c, launch_spmv(c, x, r, b, c->stream));
}

int gdsw_newton_step(gdsw_ctx* c, double* x, gdsw_solve_info* info) {
  if (!c || c->host_only || !x) return GDSW_ERR_INVALID_ARG;
  gdsw_solve_info tmp{};
  if (!info) info = &tmp;
  GDSW_TRY(c, {
    GDSW_CHECK(c->form == GDSW_FORM_SYMMETRIC && c->has_uk, GDSW_ERR_INVALID_ARG,
               "a Newton step needs the symmetric (Carreau) form and a velocity u_k");
    cudaStream_t s = c->stream;
    const int64_t n = c->mesh.n;
    if (!c->d_dn) c->d_dn = c->arena.alloc<double>(7 * 27 * int64_t(c->mesh.fluid.size()));
    if (!c->d_newton_work) c->d_newton_work = c->arena.alloc<double>(3 * n);
    double* b = c->d_newton_work;
    double* r = b + n;
    double* d = r + n;
    c->prof_gate = true;
    launch_viscosity(c, s);          // nu(u_k), D(u_k) and the Newton weights
    launch_assembly(c, s, false);    // Picard operator A(nu(u_k)) for the residual
    launch_lift(c, b, s);
    launch_spmv(c, x, r, b, s);      // R = b - A x
    launch_assembly(c, s, true);     // Jacobian J = A + Newton term
    GDSW_CUDA(cudaMemsetAsync(d, 0, 8 * n, s));
    fgmres_solve(c, r, d, info);     // J delta = R with the frozen preconditioner
    launch_axpy(x, d, n, s);         // x += delta
    launch_picard_velocity(c, x, s); // u_{k+1}
    GDSW_CHECK(info->status == GDSW_OK || info->status == GDSW_ERR_NOT_CONVERGED, info->status,
               "Newton step: the linear solve failed");
  });
}

int gdsw_picard_update(gdsw_ctx* c, const double* x) {
  if (!c || c->host_only || !x) return GDSW_ERR_INVALID_ARG;
  GDSW_TRY(c, launch_picard_velocity(c, x, c->stream));
}

int gdsw_reassemble(gdsw_ctx* c, const double* uk) {
  if (!c || c->host_only) return GDSW_ERR_INVALID_ARG;
  GDSW_TRY(c, {
    c->prof_gate = true;
    if (uk) {
      GDSW_CUDA(cudaMemcpyAsync(c->d_uk, uk, 24 * c->mesh.nnodes, cudaMemcpyHostToDevice, c->stream));
      c->has_uk = true;
    }
    {
      ProfScope ps(c, GDSW_K_VISCOSITY, 8.0 * 27 * c->mesh.fluid.size(), c->stream);
      launch_viscosity(c, c->stream);
    }
    {
      ProfScope ps(c, GDSW_K_ASSEMBLY, 8.0 * 9 * c->nnzb, c->stream);  // A only: B is viscosity-free
      launch_assembly(c, c->stream);
    }
  });
}

int gdsw_apply_local(gdsw_ctx* c, int32_t level, const double* r, double* z) {
  if (!c || c->host_only || level < 0 || level >= int(c->ld.size()) || !r || !z) return GDSW_ERR_INVALID_ARG;
  GDSW_TRY(c, local_solve(c, level, r, z, c->stream));
}

int gdsw_restrict(gdsw_ctx* c, int32_t level, const double* r, double* r0) {
  if (!c || c->host_only || level < 0 || level >= int(c->ld.size()) || !r || !r0) return GDSW_ERR_INVALID_ARG;
  GDSW_TRY(c, restrict_level(c, level, r, r0, c->stream));
}

int gdsw_prolong(gdsw_ctx* c, int32_t level, const double* x0, double* z) {
  if (!c || c->host_only || level < 0 || level >= int(c->ld.size()) || !x0 || !z) return GDSW_ERR_INVALID_ARG;
  GDSW_TRY(c, {
    const LevelDev& L = c->ld[level];
    launch_prolong(L, x0, z, c->stream);
    if (L.n0 > 0) launch_axpy_gamma(L.gu_dof, L.gu_ptr, L.gcol, L.gval, L.ngu, x0, z, c->stream);
  });
}

int gdsw_coarse_matrix(gdsw_ctx* c, int32_t l, double* host) {
  if (!c || c->host_only || !host || l < 0 || l >= c->L - 1) return GDSW_ERR_INVALID_ARG;
  GDSW_TRY(c, {
    const double* A = (l + 1 < int(c->ld.size())) ? c->ld[l + 1].A : c->coarsest_A;
    int64_t n = (l + 1 < int(c->ld.size())) ? c->ld[l + 1].n : c->n_coarsest;
    if (n > 0) GDSW_CUDA(cudaMemcpy(host, A, 8 * n * n, cudaMemcpyDeviceToHost));
  });
}

int gdsw_matrix_csr(gdsw_ctx* c, int64_t* row_ptr, int32_t* col, double* val, int64_t* nnz) {
  if (!c || c->host_only || !nnz) return GDSW_ERR_INVALID_ARG;
  GDSW_TRY(c, {
    const MeshHost& M = c->mesh;
    int64_t total = 9 * c->nnzb + 3 * c->nbt + 3 * c->nb;
    *nnz = total;
    if (row_ptr && col && val) {
      std::vector<double> v(total);
      GDSW_CUDA(cudaMemcpy(v.data(), c->d_val, 8 * total, cudaMemcpyDeviceToHost));
      const double* bt = v.data() + 9 * c->nnzb;
      const double* bb = bt + 3 * c->nbt;
      int64_t e = 0;
      row_ptr[0] = 0;
      for (int64_t I = 0; I < M.nv; ++I)
        for (int cc = 0; cc < 3; ++cc) {
          for (int32_t blk = M.a_ptr[I]; blk < M.a_ptr[I + 1]; ++blk)
            for (int d = 0; d < 3; ++d) {
              col[e] = 3 * M.a_col[blk] + d;
              val[e++] = v[int64_t(blk) * 9 + cc * 3 + d];
            }
          for (int32_t q = M.bt_ptr[I]; q < M.bt_ptr[I + 1]; ++q) {
            col[e] = int32_t(M.nu + M.bt_col[q]);
            val[e++] = bt[int64_t(q) * 3 + cc];
          }
          row_ptr[3 * I + cc + 1] = e;
        }
      for (int64_t P = 0; P < M.np; ++P) {
        for (int32_t q = M.b_ptr[P]; q < M.b_ptr[P + 1]; ++q)
          for (int d = 0; d < 3; ++d) {
            col[e] = 3 * M.b_col[q] + d;
            val[e++] = bb[int64_t(q) * 3 + d];
          }
        row_ptr[M.nu + P + 1] = e;
      }
    }
  });
}

int gdsw_viscosity_values(gdsw_ctx* c, double* host) {
  if (!c || c->host_only || !host) return GDSW_ERR_INVALID_ARG;
  GDSW_TRY(c, GDSW_CUDA(cudaMemcpy(host, c->d_nu, 8 * 27 * c->mesh.fluid.size(), cudaMemcpyDeviceToHost)));
}

int gdsw_level_dofs(gdsw_ctx* c, int32_t level, int64_t* offsets, int32_t* dofs) {
  if (!c || level < 0 || level >= int(c->lh.size()) || !offsets) return GDSW_ERR_INVALID_ARG;
  const LevelHost& H = c->lh[level];
  std::copy(H.dof_off.begin(), H.dof_off.end(), offsets);
  if (dofs) std::copy(H.dof_sorted.begin(), H.dof_sorted.end(), dofs);
  return GDSW_OK;
}

int gdsw_level_entities(gdsw_ctx* c, int32_t level, int32_t* n_entities) {
  if (!c || level < 0 || level >= int(c->lh.size()) || !n_entities) return GDSW_ERR_INVALID_ARG;
  *n_entities = c->lh[level].cs.n_entities;
  return GDSW_OK;
}

int64_t gdsw_kernel_launches(void) { return launch_counter(); }

int gdsw_plan_bytes(const gdsw_ctx* c, int32_t level, int32_t direction, int32_t k, double* bytes) {
  if (!c || c->host_only || !bytes || level < 0 || level >= int(c->ld.size())) return GDSW_ERR_INVALID_ARG;
  if (direction == 2) {
    if (k != 0) return GDSW_ERR_INVALID_ARG;
    *bytes = c->ld[level].red_bytes;
    return GDSW_OK;
  }
  if (direction != 0 && direction != 1) return GDSW_ERR_INVALID_ARG;
  const std::vector<double>& v = direction == 0 ? c->ld[level].fwd_bytes : c->ld[level].bwd_bytes;
  if (k < 0 || k >= int(v.size())) return GDSW_ERR_INVALID_ARG;
  *bytes = v[k];
  return GDSW_OK;
}

int gdsw_sweep_wait_selftest(gdsw_ctx* c) {
  if (!c || c->host_only || c->ld.empty() || c->ld[0].sweep.nitems == 0) return GDSW_ERR_INVALID_ARG;
  LevelDev& L = c->ld[0];
  cudaStream_t s = c->stream;
  DevArena tmp(s);
  unsigned flag = 0;
  try {
    std::vector<SweepItem> items(L.sweep.nitems);
    GDSW_CUDA(cudaMemcpyAsync(items.data(), L.sweep.d_items, sizeof(SweepItem) * items.size(), cudaMemcpyDeviceToHost, s));
    GDSW_CUDA(cudaStreamSynchronize(s));
    size_t q = 0;
    while (q < items.size() && items[q].wait0 < 0) ++q;
    GDSW_CHECK(q < items.size(), GDSW_ERR_INVALID_ARG, "level-1 sweep has no dependency to wait for");
    items[q].need0 += 1;  // one more than its producers will ever signal
    SweepPlan P = L.sweep;
    P.d_items = tmp.upload(items, s);
    if (L.prec == GDSW_FP64)
      launch_sweep<double, double>(static_cast<const double*>(L.fac), static_cast<double*>(L.vec), P, c->d_sweep_flag,
                                   L.sym_T, s);
    else if (L.prec == GDSW_FP32)
      launch_sweep<float, float>(static_cast<const float*>(L.fac), static_cast<float*>(L.vec), P, c->d_sweep_flag,
                                 L.sym_T, s);
    else
      launch_sweep<__nv_bfloat16, float>(static_cast<const __nv_bfloat16*>(L.fac), static_cast<float*>(L.vec), P,
                                         c->d_sweep_flag, L.sym_T, s);
    GDSW_CUDA(cudaMemcpyAsync(&flag, c->d_sweep_flag, sizeof(flag), cudaMemcpyDeviceToHost, s));
    GDSW_CUDA(cudaMemsetAsync(c->d_sweep_flag, 0, sizeof(unsigned), s));
    GDSW_CUDA(cudaStreamSynchronize(s));
  } catch (const gdsw::Error& e) {
    tmp.free_all();
    c->err = e.msg;
    return e.code;
  }
  tmp.free_all();
  if (!flag) {
    c->err = "gdsw_sweep_wait_selftest: the unsatisfiable wait did not report a timeout";
    return GDSW_ERR_CUDA;
  }
  c->err = "persistent local sweep: a dependency wait exceeded its time limit (self-test)";
  return GDSW_ERR_TIMEOUT;
}

int gdsw_set_local_sweep(gdsw_ctx* c, int32_t persistent, int32_t ctas_per_sm, int32_t tile_rows) {
  if (!c || c->host_only || ctas_per_sm < 0) return GDSW_ERR_INVALID_ARG;
  if (tile_rows != 0 && tile_rows != 32 && tile_rows != 64 && tile_rows != 128) return GDSW_ERR_INVALID_ARG;
  if (c->apply_graph) {
    c->err = "gdsw_set_local_sweep: the apply is already captured in a CUDA graph (use_graph)";
    return GDSW_ERR_INVALID_ARG;
  }
  GDSW_TRY(c, {
    for (size_t l = 0; l < c->ld.size(); ++l) {
      LevelDev& L = c->ld[l];
      L.persistent = persistent != 0;
      if (tile_rows != 0 && tile_rows != L.fwd.rows_per_tile) {
        L.fwd.rows_per_tile = tile_rows;
        build_local_plan(c, c->lh[l].loc, L);
      }
      resize_sweep(L, ctas_per_sm);
    }
  });
}

int gdsw_profile_enable(gdsw_ctx* c, int32_t on) {
  if (!c) return GDSW_ERR_INVALID_ARG;
  // on = 0: off; on = k >= 1: time every k-th preconditioner apply and the work after it
  c->prof.enabled = on ? 1 : 0;
  c->prof_stride = on > 1 ? on : 1;
  c->apply_count = 0;
  c->prof_gate = true;
  return GDSW_OK;
}

int gdsw_profile_read(gdsw_ctx* c, gdsw_profile* p) {
  if (!c || !p) return GDSW_ERR_INVALID_ARG;
  GDSW_TRY(c, {
    prof_collect(c);
    *p = c->prof;
  });
}

int gdsw_profile_reset(gdsw_ctx* c) {
  if (!c) return GDSW_ERR_INVALID_ARG;
  GDSW_TRY(c, {
    prof_collect(c);
    int en = c->prof.enabled;
    c->prof = gdsw_profile{};
    c->prof.enabled = en;
  });
}

}  // extern "C"
