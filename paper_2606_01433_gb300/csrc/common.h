// Internal definitions shared by the translation units of libgdsw.so.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/gdsw.h"

namespace gdsw {

// ------------------------------------------------------------------ errors
struct Error {
  int code;
  std::string msg;
};

#define GDSW_CUDA(call)                                                                      \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      throw ::gdsw::Error{e_ == cudaErrorMemoryAllocation ? GDSW_ERR_OOM : GDSW_ERR_CUDA,    \
                          std::string(#call) + ": " + cudaGetErrorString(e_)};              \
  } while (0)

#define GDSW_CHECK(cond, code, text)                                                         \
  do {                                                                                       \
    if (!(cond)) throw ::gdsw::Error{(code), (text)};                                        \
  } while (0)

// every kernel launch of the library is followed by check_launch, which also counts it
std::atomic<int64_t>& launch_counter();
inline void check_launch(const char* what) {
  ++launch_counter();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw Error{GDSW_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e)};
}

// ------------------------------------------------------------------ overlapped launch chains
// A launch made with programmatic dependent launch may have CTAs resident while the previous
// kernel of its stream drains.  Every kernel launched that way calls dep_release() (its own
// dependents may start) and dep_wait() (the previous grid has completed and its writes are
// visible) before it reads anything the previous kernels wrote or writes anything they read;
// before the wait it may only read data that no kernel of the stream writes (factors, plans,
// the operator); the wait makes the previous grid's writes visible to this grid.  A kernel
// that follows a wait on another stream's event is launched in plain order: the dependency
// wait covers only the previous grid of its own stream.  Both instructions do nothing in a
// launch made without the attribute.
// g_launch_overlap (gdsw_set_launch_overlap) switches the attribute off process-wide.
extern bool g_launch_overlap;
#ifdef __CUDACC__
__device__ __forceinline__ void dep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

template <typename... KArgs, typename... Args>
inline void launch_chained(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                           Args... args) {
  if (!g_launch_overlap) {
    kernel<<<grid, block, smem, s>>>(args...);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, KArgs(args)...);
  if (e != cudaSuccess) throw Error{GDSW_ERR_CUDA, std::string("chained launch: ") + cudaGetErrorString(e)};
}
#endif

// ------------------------------------------------------------------ device memory
// Stream-ordered when built with a stream (cudaMallocAsync / cudaFreeAsync on that stream):
// freeing then never waits for the whole device, so contexts that set up, solve and tear down
// on different streams (the solve server's slots) do not stall one another.  Memory of an
// arena may only be used by work ordered after its allocation on that stream and freed after
// the last such work.
struct DevArena {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
  bool ordered = false;
  DevArena() = default;
  explicit DevArena(cudaStream_t s) : stream(s), ordered(true) {}
  template <typename T>
  T* alloc(size_t n) {
    if (n == 0) n = 1;
    void* p = nullptr;
    if (ordered)
      GDSW_CUDA(cudaMallocAsync(&p, n * sizeof(T), stream));
    else
      GDSW_CUDA(cudaMalloc(&p, n * sizeof(T)));
    ptrs.push_back(p);
    bytes += n * sizeof(T);
    return static_cast<T*>(p);
  }
  template <typename T>
  T* upload(const std::vector<T>& v, cudaStream_t s) {
    T* p = alloc<T>(v.size());
    if (!v.empty()) GDSW_CUDA(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return p;
  }
  void free_one(void* p) {
    if (ordered)
      cudaFreeAsync(p, stream);
    else
      cudaFree(p);
  }
  void release(void* p) {
    for (auto& q : ptrs)
      if (q == p) {
        free_one(q);
        q = nullptr;
      }
  }
  void free_all() {
    for (void* p : ptrs)
      if (p) free_one(p);
    ptrs.clear();
    bytes = 0;
  }
};

inline size_t elem_size(int prec) { return prec == GDSW_FP64 ? 8 : (prec == GDSW_FP32 ? 4 : 2); }
inline int64_t pad8(int64_t x) { return (x + 7) & ~int64_t(7); }

// ------------------------------------------------------------------ device task descriptors
// One dense matrix-vector product y[r] = base[r] + alpha * sum_c M[r, c] x[c] over rows of a
// row-major block M (leading dimension ld, padded with zeros to a multiple of 8 columns).
struct GemvTask {
  int64_t mat;      // element offset of M in the factor buffer
  int64_t x;        // element offset of x in the vector buffer
  int64_t y;        // element offset of y
  int64_t base;     // element offset of base (or -1: zero)
  int32_t rows, cols, ld;  // kind 1: rows = cols = block size, ld = number of tiles per side
  float alpha;
  int32_t kind;     // 0: dense row-major rows; 1: symmetric block stored as packed upper tiles
  int32_t pad_;
  int64_t part;     // kind 1: element offset of the partial sums (nt x nt x T) in the vector buffer
};
// A CTA's share of a GEMV launch: rows [row0, row0 + nrows) of task `task`.
struct GemvTile {
  int32_t task, row0;
};

// Batched GEMM C = alpha op(A) op(B) + beta C (row-major, element offsets into buffers).
struct GemmTask {
  int64_t a, b, c;
  int32_t M, N, K, lda, ldb, ldc;
  int32_t ta, tb;   // 1 = transposed operand
  double alpha, beta;
};

// Batched dense inverse (in place) of square n x n blocks with leading dimension ld.
struct InvTask {
  int64_t a;        // element offset of the matrix
  int32_t n, ld;
  int32_t id;       // index into the status / scratch arrays
};

// ------------------------------------------------------------------ host symbolic structures
// A batch of block-tridiagonal local problems: dof lists in slab order, slab sizes, the
// number of back-coupled dofs (those coupled to the previous slab, ordered first) and the
// offsets of the LDL^T blocks Sinv_k (s_k x s_k) and G_k (m_k x s_{k-1}); the
// super-diagonal blocks of the symmetric factorisation are the transposes G_{k+1}^T, so no
// W_k block is stored (fW = -1).
struct SlabSet {
  int nsub = 0;
  int Kmax = 0;
  std::vector<int> K;
  std::vector<std::vector<int>> s, m;
  std::vector<int64_t> voff;                 // subdomain offset in the concatenated local vector
  std::vector<std::vector<int64_t>> soff;    // slab offset relative to voff
  std::vector<std::vector<int64_t>> fS, fG, fW;
  std::vector<std::vector<int>> ldS, ldG, ldW;
  int64_t nvec = 0, nfac = 0;
  std::vector<int32_t> gdof;                 // local position -> global dof of the level
  int64_t max_local = 0;
  void layout();                             // fills voff/soff/f*/ld*/nvec/nfac from s, m, K
};

// A coarse space towards the next level, in the form the apply uses on every level:
// interior blocks Phi_I,J (stored transposed, c_J x n_IJ) per part, plus the interface map.
struct CoarseSpace {
  int n = 0;        // size of this level
  int n0 = 0;       // coarse size
  int nparts = 0;
  std::vector<int32_t> idofs;       // concatenated interior dofs per part (slab order for level 1)
  std::vector<int64_t> ioff;        // per part offset into idofs (nparts + 1)
  std::vector<int32_t> cols;        // concatenated coarse columns per part (ascending)
  std::vector<int64_t> coff;        // per part offset into cols (nparts + 1)
  std::vector<int32_t> gdofs, gcol; // Phi_Gamma entries: interface dof (ascending), coarse column
  std::vector<double> gval;         //   and value (1 for translations and pressure constants)
  std::vector<int32_t> gu_dof, gu_ptr;  // the distinct interface dofs and their entry ranges
  std::vector<double> rg_val;       // values of the rg lists below
  // restriction reduce lists per coarse dof: positions in the concatenated per-part
  // result buffer (offset coff[J] + local column) and interface dofs
  std::vector<int32_t> rr_ptr, rr_pos, rg_ptr, rg_dof;
  // coarse nodes of the next level: sharing set (parts of this level), dofs, modes
  std::vector<std::vector<int>> cn_set;
  std::vector<std::vector<int>> cn_dofs, cn_modes;
  int n_entities = 0;
};

struct LevelHost {
  int n = 0, N = 0;
  SlabSet loc;                      // overlapping local problems
  std::vector<int32_t> sc_ptr, sc_pos;   // scatter lists per dof of the level
  std::vector<double> sc_w;              // weights (1/multiplicity or 1)
  std::vector<int64_t> dof_off;     // sorted overlapping dof lists (for gdsw_level_dofs)
  std::vector<int32_t> dof_sorted;
  CoarseSpace cs;
  SlabSet inter;                    // level 1: interior problems (slab order)
};

struct MeshHost {
  int nx, ny, nz;
  double h, origin[3];
  int NX, NY, NZ;
  int64_t nnodes;
  std::vector<uint8_t> mask, tags;
  std::vector<double> g;
  std::vector<int32_t> felem;       // element -> fluid index or -1
  std::vector<int32_t> fluid;       // fluid index -> element
  std::vector<int32_t> vidx, pidx;  // node -> free velocity / pressure index, -1
  std::vector<int32_t> vnode, pnode;// index -> node
  std::vector<uint8_t> active;
  int64_t nv = 0, np = 0, n = 0, nu = 0;
  bool pdisc = false;                    // P1-disc pressure: rows 4 f + k per fluid element f
  // patterns
  std::vector<int32_t> a_ptr, a_col;     // velocity node rows x velocity node cols
  std::vector<int32_t> bt_ptr, bt_col;   // velocity node rows x pressure cols
  std::vector<int32_t> b_ptr, b_col;     // pressure rows x velocity node cols
  std::vector<int32_t> bt2b;             // BT entry -> B entry with the same value
  std::vector<int32_t> a_diag, a_tpos;   // position of block (I,I); position of block (J,I) for (I,J)
  std::vector<int32_t> ad_ptr, ad_col;   // velocity rows x Dirichlet nodes with g != 0 (node ids)
  std::vector<int32_t> bd_ptr, bd_col;   // pressure rows x Dirichlet nodes with g != 0
  // assembly work units: one (upper block (I, J >= I), shared fluid element) pair each, listed
  // block by block (elements in increasing index); packed fluid element << 10 | a << 5 | b
  // with a, b the local Q2 node numbers of I and J in that element
  std::vector<int32_t> asm_uoff;         // per block: first unit (lower blocks own none), nnzb + 1
  std::vector<uint32_t> asm_unit;
  std::vector<int32_t> asm_cta;          // first block of each assembly CTA (<= 256 units), + nnzb
  // sliced copy of the velocity rows for the SpMV (32 rows per slice, rows sorted by length
  // inside windows of 1024 rows so that a slice's rows have near-equal lengths): slot
  // j * 32 + lane of slice s holds the j-th block (or B^T entry) of the slice's lane-th row
  std::vector<int32_t> sell_row;         // nslices * 32: velocity row or -1
  std::vector<int64_t> sell_aoff, sell_boff;  // nslices + 1: first block / B^T slot of each slice
  std::vector<int32_t> sell_acol, sell_asrc;  // per block slot: column node, source block (-1: pad)
  std::vector<int32_t> sell_bcol, sell_bsrc;  // per B^T slot: pressure column, source entry (-1: pad)
  bool shares_element(int64_t a, int64_t b) const;
  void coords(int64_t node, int& i, int& j, int& k) const {
    i = int(node % NX);
    j = int((node / NX) % NY);
    k = int(node / (int64_t(NX) * NY));
  }
};

// ------------------------------------------------------------------ device-side level data
struct GemvPlan {
  std::vector<int> launch_task_off, launch_tile_off;  // nlaunch + 1
  GemvTask* d_tasks = nullptr;
  GemvTile* d_tiles = nullptr;
  int rows_per_tile = 32;
  bool transposed = false;      // tiles are 256-column blocks of y = M^T x
  int nlaunch() const { return int(launch_task_off.size()) - 1; }
};

// One item of a persistent level sweep: a tile of one task, the per-slab counters it waits
// for (index into the counter array, value to reach; -1 = none) and the counter it bumps.
enum { SWEEP_ROWS = 0, SWEEP_SYM = 1, SWEEP_REDUCE = 2, SWEEP_COLS = 3 };
struct SweepItem {
  int32_t op, task, arg, signal;
  int32_t wait0, need0, wait1, need1;
};
struct SweepPlan {
  SweepItem* d_items = nullptr;
  GemvTask* d_tasks = nullptr;   // forward, backward and reduction tasks of the level
  unsigned* d_ctr = nullptr;     // [0] = claim counter, then 4 counters per slab
  int nitems = 0, nctr = 0, xs_elems = 0, grid = 0, ctas_per_sm = 0, max_per_sm = 0;
  int G = 1;                     // row groups of 32 per forward tile
  size_t smem = 0;
};
constexpr unsigned long long kSweepWaitLimitNs = 1000000000ull;  // 1 s per wait

struct LevelDev {
  int n = 0, N = 0, prec = GDSW_FP64;
  // local problems
  void* fac = nullptr;          // factors in storage precision
  int64_t nfac = 0, nvec = 0;
  int32_t* gdof = nullptr;
  GemvPlan fwd, bwd;            // forward launches (Sinv, G) and backward launches (G^T)
  SweepPlan sweep;              // the same tiles as one persistent launch
  bool persistent = false;      // local solve as the persistent launch (else one launch per slab step)
  double tuned_ms = 0;          // autotuned local-solve time (0: not tuned)
  void* vec = nullptr;          // local vector workspace (2 * nvec, compute precision)
  int32_t *sc_ptr = nullptr, *sc_pos = nullptr;
  double* sc_w = nullptr;
  // coarse space
  int n0 = 0, phi_prec = GDSW_FP64;
  int32_t *idofs = nullptr, *cols = nullptr, *gdofs = nullptr, *gcol = nullptr;
  int32_t *gu_dof = nullptr, *gu_ptr = nullptr;  // Phi_Gamma entries grouped by interface dof
  double* gval = nullptr;                        // Phi_Gamma values
  double* rg_val = nullptr;
  int64_t nidofs = 0, ncols = 0, ngamma = 0, ngu = 0;
  void* phiT = nullptr;         // concatenated Phi_I^T blocks
  // restriction partials: per (part J, row j) the nt_J tile partials at part_poff[J] + j nt_J + t;
  // per cols entry q (row j of part J) the start and count of its partials
  double* partial = nullptr;
  int64_t *part_poff = nullptr, *q_start = nullptr;
  int32_t *part_ntiles = nullptr, *q_count = nullptr, *pro_tile_rank = nullptr;
  int32_t *pro_part = nullptr;  // per prolongation tile: part
  int64_t* pro_meta = nullptr;  // per part: phiT offset, ld, idofs offset, n_I, cols offset, c
  int n_pro_tiles = 0;
  int max_c = 0;
  int max_ld_fwd = 0;
  std::vector<int> fwd_ld, bwd_ld;  // largest input length per launch
  int32_t *pro_tile_part = nullptr, *pro_tile_col0 = nullptr;
  int32_t *rr_ptr = nullptr, *rr_pos = nullptr, *rg_ptr = nullptr, *rg_dof = nullptr;
  // level vectors (FP64)
  double* r = nullptr;          // this level's right-hand side (coarse levels)
  double* z = nullptr;          // this level's result (coarse levels)
  double* x0 = nullptr;         // next-level solution (n0)
  double* r0 = nullptr;         // restricted residual (n0)
  double* zc = nullptr;         // local-branch result when the branches overlap
  // dense coarse operator of THIS level (levels >= 2), FP64 row-major
  double* A = nullptr;
  std::vector<double> fwd_bytes, bwd_bytes;  // algorithmic bytes of each GEMV launch
  // storage layout of the factors: per (part, slab) flattened in part-major order
  std::vector<int64_t> pS, pG;  // offsets of S_k^{-1} (packed tiles or dense) and of G_k
  std::vector<uint8_t> psym;    // S_k^{-1} stored as packed symmetric tiles
  int sym_T = 128;
  int64_t npart = 0;            // partial-sum entries behind the 2 nvec local vectors
  GemvPlan red;                 // reduction of the symmetric partial sums (one launch)
  double red_bytes = 0;
  double minpiv = 0;            // smallest pivot magnitude met by the local factorisation
  double local_bytes = 0;       // algorithmic bytes of one local-solve sweep pair
  double phi_bytes = 0;         // bytes of the stored Phi_I^T blocks
};

}  // namespace gdsw

// ------------------------------------------------------------------ the context
struct gdsw_ctx {
  std::string err;
  bool host_only = false;           // created by gdsw_analyze: no device state
  int device = -1;                  // CUDA device current at set-up (owns every device buffer)
  // preconditioner attached from outside (a multigrid V-cycle over this context's grid), or null
  void (*ext_precond)(void* data, const double* r, double* z, cudaStream_t s) = nullptr;
  void* ext_data = nullptr;
  bool host_ready = false;          // host symbolic structures built
  bool capturing = false;           // inside CUDA-graph capture (no profiling events)
  int prof_stride = 1;              // time every prof_stride-th apply (and the work after it)
  int64_t apply_count = 0;
  bool prof_gate = true;
  double apply_bytes = 0;           // algorithmic bytes of one preconditioner apply
  int64_t est_device_bytes = 0;
  cudaStream_t stream = nullptr, stream2 = nullptr;
  bool own_stream = false;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  gdsw_options opt{};
  int L = 2;
  gdsw::DevArena arena;
  gdsw::MeshHost mesh;
  std::vector<gdsw::LevelHost> lh;
  std::vector<gdsw::LevelDev> ld;
  // viscosity parameters
  int form = GDSW_FORM_GRADIENT;
  double nu0 = 1, nu_inf = 0, lam = 0, ncar = 1;
  bool has_uk = false;
  // device mesh / matrix
  double* d_uk = nullptr;
  double* d_nu = nullptr;           // nu[fluid element][27]
  double* d_dn = nullptr;           // Newton linearisation: D(u_k) and N per Gauss point (7 values), or null
  double* d_newton_work = nullptr;  // Newton step: lifted b, residual, increment (3 n)
  uint8_t* d_mask = nullptr;
  int32_t* d_fluid = nullptr;       // fluid index -> element
  int32_t* d_felem = nullptr;
  int32_t *d_vnode = nullptr, *d_pnode = nullptr, *d_vidx = nullptr;
  int32_t *d_a_ptr = nullptr, *d_a_col = nullptr, *d_bt_ptr = nullptr, *d_bt_col = nullptr;
  int32_t *d_a_diag = nullptr, *d_a_tpos = nullptr;  // diagonal block of each row, transpose map
  int32_t *d_asm_cta = nullptr, *d_asm_uoff = nullptr;  // assembly work units (see MeshHost)
  uint32_t* d_asm_unit = nullptr;
  int32_t *d_sell_row = nullptr, *d_sell_acol = nullptr, *d_sell_asrc = nullptr;  // sliced SpMV copy
  int32_t *d_sell_bcol = nullptr, *d_sell_bsrc = nullptr;
  int64_t *d_sell_aoff = nullptr, *d_sell_boff = nullptr;
  double *d_sell_aval = nullptr, *d_sell_btval = nullptr;
  int64_t n_sell_slices = 0;
  int32_t *d_b_ptr = nullptr, *d_b_col = nullptr, *d_bt2b = nullptr;
  int32_t *d_ad_ptr = nullptr, *d_ad_col = nullptr, *d_bd_ptr = nullptr, *d_bd_col = nullptr;
  int32_t* d_lift_rows = nullptr;   // rows (velocity node, or nv + pressure node) with a Dirichlet neighbour
  int64_t n_lift_rows = 0;
  bool b_assembled = false;         // B does not depend on the viscosity: assembled once
  unsigned* d_sweep_flag = nullptr; // set by a persistent sweep whose wait ran out
  double* d_gdir = nullptr;         // Dirichlet datum, 3 per node
  void* d_tables = nullptr;         // RefTables
  double* d_val = nullptr;          // [A blocks (9 per block) | BT (3 per entry) | B (3 per entry)]
  int64_t nnzb = 0, nbt = 0, nb = 0;
  double* d_coarsest_inv = nullptr; // inverse of A_0^(L), FP64
  int n_coarsest = 0;
  int ld_coarsest = 8;
  gdsw::GemvPlan coarsest_plan;
  double* coarsest_A = nullptr;     // A_0^(L) itself (kept for inspection)
  double coarsest_minpiv = 0;
  double *d_hb = nullptr, *d_hx = nullptr;  // device staging for gdsw_solve_host
  double spmv_bytes() const {
    return 76.0 * nnzb + 28.0 * double(nbt + nb) + 16.0 * double(mesh.n) + 8.0 * double(mesh.nv + mesh.np);
  }
  // FGMRES workspace
  int m_alloc = 0;
  double *d_V = nullptr, *d_Z = nullptr, *d_w = nullptr, *d_H = nullptr, *d_gvec = nullptr;
  double *d_cs = nullptr, *d_sn = nullptr, *d_part = nullptr, *d_scal = nullptr, *d_y = nullptr;
  double h_scal[8] = {0};           // host mirror of a few scalars
  int n_part_blocks = 0;
  int* d_status = nullptr;          // device error word
  // CUDA graph of the apply
  cudaGraphExec_t apply_graph = nullptr;
  const double* graph_r = nullptr;
  double* graph_z = nullptr;
  double *d_graph_r = nullptr, *d_graph_z = nullptr;
  // profiling
  gdsw_profile prof{};
  std::vector<cudaEvent_t> ev_pool;
  struct Pending { int group; cudaEvent_t a, b; double bytes; };
  std::vector<Pending> pending;
  double bytes_group[12] = {0};
  gdsw_sizes_info sizes{};
  double setup_ms[6] = {0};
};

namespace gdsw {
// CUDA-event timing of one kernel group on one stream when profiling is enabled; the pair
// is read back by gdsw_profile_read together with the group's algorithmic bytes.
struct ProfScope {
  gdsw_ctx* c;
  int group;
  double bytes;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  bool on = false;
  ProfScope(gdsw_ctx* c_, int g, double by, cudaStream_t st) : c(c_), group(g), bytes(by), s(st) {
    on = c->prof.enabled && c->prof_gate && !c->capturing;
    if (!on) return;
    a = take();
    b = take();
    cudaEventRecord(a, s);
  }
  cudaEvent_t take() {
    if (!c->ev_pool.empty()) {
      cudaEvent_t e = c->ev_pool.back();
      c->ev_pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  ~ProfScope() {
    if (!on) return;
    cudaEventRecord(b, s);
    c->pending.push_back({group, a, b, bytes});
  }
};
}  // namespace gdsw
