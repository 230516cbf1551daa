// Batched FP32 GEMM of the set-up on the fifth-generation tensor cores (tcgen05.mma,
// kind::tf32), with operands staged by TMA (cp.async.bulk.tensor) and the accumulator in
// tensor memory.  It carries the dense contractions of the local factorisation (arXiv
// 2606.01433, Section 2.1: the local saddle-point matrices A_i, factored here as block LDL^T
// slabs, G_k = B_k S_{k-1}^{-1} and S_k = A_kk - G_k B_k^T) and of the coarse basis
// (Phi_I = -A_II^{-1} A_IGamma Phi_Gamma with many right-hand sides, Section 2.1).
//
// FP32 accuracy from TF32 inputs (3xTF32): every operand entry is split as x = hi + lo with
// hi = x rounded to TF32 and lo = x - hi (exact in FP32); the product is
// A_hi B_hi + A_hi B_lo + A_lo B_hi (the lo*lo term is below FP32 rounding), which is one TF32
// GEMM with the K dimension tripled: A' = [A_hi | A_hi | A_lo], B' = [B_hi ; B_lo ; B_hi].
// A split pass writes A' and B'^T K-major (every K section zero padded to a multiple of 32)
// for all tasks of a batch, stacked by rows; one TMA descriptor per operand covers the batch.
//
// The GEMM kernel: one 128 x 128 output tile per CTA, 6 warps.  Warp 0 (one lane) issues the
// TMA loads of a 6-stage ring (32 K-columns of A and B per stage, 128-byte swizzle), warp 1
// owns the tensor-memory allocation and (one lane) issues four 128x128x8 MMAs per stage, each
// stage released by tcgen05.commit to its "empty" barrier; warps 2-5 read the accumulator
// (tcgen05.ld, one TMEM lane quarter each) and write C = alpha acc + beta C.  Every
// mbarrier wait is bounded: past the limit the kernel sets an error word, every role stops,
// the producer waits (bounded) for the loads it issued, and the tensor memory is freed.
#include <cuda.h>

#include "common.h"
#include "kernels.h"

namespace gdsw {

namespace tc {

constexpr int BM = 128, BN = 128, BK = 32, STAGES = 6;
constexpr int STAGE_BYTES = (BM + BN) * BK * 4;  // 32 KiB: A and B slices of one stage
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr uint32_t WAIT_LIMIT = 1u << 24;         // polls before a wait gives up (>= ~1 s)

struct Task {
  float* c;
  int64_t ldc;
  int32_t M, N;
  int32_t arow, brow;   // first row of the task's A' / B'^T in the stacked operands
  int32_t kblocks;      // 3 Kp / 32
  float alpha, beta;
};
struct Tile {
  int32_t task, m0, n0, pad;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the phase of the given parity; false (and the error word set) on expiry
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, unsigned* err) {
  for (uint32_t i = 0; i < WAIT_LIMIT; ++i) {
    if (mbar_try(b, parity)) return true;
    if (i >= 64) __nanosleep(64);
    if ((i & 1023u) == 0 && *(volatile unsigned*)err) return false;
  }
  atomicExch(err, 1u);
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
  const uint64_t addr = smem_u32(p);
  uint64_t d = 0;
  d |= (addr >> 4) & 0x3FFFull;          // start address
  d |= uint64_t(1) << 16;                // leading byte offset (unused by swizzled K-major)
  d |= uint64_t(1024 >> 4) << 32;        // stride byte offset: next 8-row group
  d |= uint64_t(1) << 46;                // descriptor version of this architecture
  d |= uint64_t(2) << 61;                // 128-byte swizzle
  return d;
}

// instruction descriptor: D FP32, A and B TF32, both K-major, M = 128, N = 128
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(BN >> 3) << 17) | (uint32_t(BM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(IDESC), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__global__ void __launch_bounds__(192, 1) k_tc_gemm(const __grid_constant__ CUtensorMap tmA,
                                                    const __grid_constant__ CUtensorMap tmB,
                                                    const Task* __restrict__ tasks, const Tile* __restrict__ tiles,
                                                    unsigned* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;                                  // STAGES x [128 rows][32 floats], swizzled
  uint8_t* sB = smem + STAGES * BM * BK * 4;           // STAGES x [128 rows][32 floats], swizzled
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);

  const Tile tile = tiles[blockIdx.x];
  const Task T = tasks[tile.task];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = T.kblocks;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(uint32_t(BN)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer: TMA loads of the A' and B'^T slices of every K block
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      if (kb >= STAGES && !mbar_wait(empty + s, ((kb / STAGES) - 1) & 1, err)) break;
      mbar_expect_tx(full + s, STAGE_BYTES);
      tma_load_2d(sA + s * BM * BK * 4, &tmA, kb * BK, T.arow + tile.m0, full + s);
      tma_load_2d(sB + s * BN * BK * 4, &tmB, kb * BK, T.brow + tile.n0, full + s);
      issued = kb + 1;
    }
    // every issued load has landed before the CTA may exit (immediate on the normal path)
    for (int kb = issued > STAGES ? issued - STAGES : 0; kb < issued; ++kb)
      mbar_wait(full + (kb % STAGES), (kb / STAGES) & 1, err);
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: four K = 8 steps per stage, stage released when its MMAs complete
    bool ok = true;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      if (!mbar_wait(full + s, (kb / STAGES) & 1, err)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t da = smem_desc(sA + s * BM * BK * 4), db = smem_desc(sB + s * BN * BK * 4);
#pragma unroll
      for (int k = 0; k < BK / 8; ++k)  // +32 bytes per K step inside the 128-byte swizzle row
        mma_tf32(tmem, da + uint64_t(2 * k), db + uint64_t(2 * k), (kb > 0 || k > 0) ? 1u : 0u);
      mma_commit(empty + s);
    }
    if (ok) mma_commit(done);
  } else if (warp >= 2) {
    // epilogue: TMEM lanes 32 (warp % 4) .. +31 hold rows of the tile, columns 0..127; one lane
    // waits, so the warp stays converged for the .sync.aligned tensor-memory loads
    int ok = 0;
    if (lane == 0) ok = mbar_wait(done, 0, err) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int q = warp & 3;
      const int row = tile.m0 + 32 * q + lane;
      float* crow = T.c + int64_t(row) * T.ldc;
      for (int c0 = 0; c0 < BN; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + (uint32_t(32 * q) << 16) + uint32_t(c0), v);
        if (row < T.M) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = tile.n0 + c0 + j;
            if (col < T.N) crow[col] = T.beta != 0.f ? fmaf(T.alpha, v[j], T.beta * crow[col]) : T.alpha * v[j];
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(uint32_t(BN)));
  }
}

// ---- split pass: x = hi + lo, written K-major into the stacked operand
struct SplitTask {
  const float* x;
  int64_t ldx;
  int32_t rows, K, Kp, trans;  // logical rows x K matrix; trans: element (r, k) at x[k ldx + r]
  int64_t row0;                // first row in the stacked operand
};

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// order 0 (A'): sections (hi, hi, lo); order 1 (B'^T): sections (hi, lo, hi)
__global__ void __launch_bounds__(256) k_tc_split(const SplitTask* __restrict__ tasks, float* __restrict__ out,
                                                  int64_t ldo, int order) {
  __shared__ float t[32][33];
  const SplitTask S = tasks[blockIdx.z];
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  if (r0 >= S.rows || k0 >= S.Kp) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int i = ty; i < 32; i += 8) {
    float v = 0.f;
    if (S.trans) {  // coalesced along r
      const int k = k0 + i, r = r0 + tx;
      if (k < S.K && r < S.rows) v = S.x[int64_t(k) * S.ldx + r];
      t[tx][i] = v;
    } else {        // coalesced along k
      const int r = r0 + i, k = k0 + tx;
      if (k < S.K && r < S.rows) v = S.x[int64_t(r) * S.ldx + k];
      t[i][tx] = v;
    }
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int r = r0 + i, k = k0 + tx;
    if (r >= S.rows || k >= S.Kp) continue;
    const float v = t[i][tx];
    const float hi = tf32_round(v), lo = v - hi;
    float* o = out + (S.row0 + r) * ldo + k;
    o[0] = hi;
    o[S.Kp] = order == 0 ? hi : lo;
    o[2 * S.Kp] = order == 0 ? lo : hi;
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    GDSW_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    GDSW_CHECK(q == cudaDriverEntryPointSuccess && p, GDSW_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// rows x width FP32 row-major, 128-byte rows of the box (32 floats) x 128 rows, zero fill
static CUtensorMap make_map(float* base, int64_t rows, int64_t width) {
  CUtensorMap m;
  cuuint64_t dims[2] = {cuuint64_t(width), cuuint64_t(rows)};
  cuuint64_t strides[1] = {cuuint64_t(width) * 4};
  cuuint32_t box[2] = {uint32_t(BK), uint32_t(BM)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  GDSW_CHECK(r == CUDA_SUCCESS, GDSW_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string(int(r)));
  return m;
}

}  // namespace tc

// Tasks as for run_gemm (C = alpha op(A) op(B) + beta C, FP32, row-major); K >= 1.  The
// stacked split operands live in a local stream-ordered arena freed before returning.
void run_gemm_tc(const std::vector<GemmTaskP>& in, cudaStream_t s) {
  using namespace tc;
  if (in.empty()) return;
  static bool attr = false;
  if (!attr) {
    GDSW_CUDA(cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    attr = true;
  }
  int Kmax = 0, Mmax = 0, Nmax = 0;
  int64_t arows = 0, brows = 0;
  for (const GemmTaskP& g : in) {
    GDSW_CHECK(g.M > 0 && g.N > 0 && g.K > 0, GDSW_ERR_INVALID_ARG, "tensor-core GEMM: empty task");
    Kmax = std::max(Kmax, g.K);
    Mmax = std::max(Mmax, g.M);
    Nmax = std::max(Nmax, g.N);
  }
  const int KpMax = (Kmax + BK - 1) / BK * BK;
  const int64_t W = 3 * int64_t(KpMax);  // stacked operand width (floats); rows 128-byte aligned
  std::vector<SplitTask> sa, sb;
  std::vector<Task> tasks;
  std::vector<Tile> tiles;
  for (const GemmTaskP& g : in) {
    const int Kp = (g.K + BK - 1) / BK * BK;
    sa.push_back({static_cast<const float*>(g.a), g.lda, g.M, g.K, Kp, g.ta, arows});
    // B'^T row n = column n of op(B): element (n, k) = op(B)(k, n)
    sb.push_back({static_cast<const float*>(g.b), g.ldb, g.N, g.K, Kp, g.tb ? 0 : 1, brows});
    const int id = int(tasks.size());
    tasks.push_back({static_cast<float*>(g.c), g.ldc, g.M, g.N, int32_t(arows), int32_t(brows), 3 * Kp / BK,
                     float(g.alpha), float(g.beta)});
    for (int m0 = 0; m0 < g.M; m0 += BM)
      for (int n0 = 0; n0 < g.N; n0 += BN) tiles.push_back({id, m0, n0, 0});
    arows += g.M;
    brows += g.N;
  }
  GDSW_CHECK(arows < (int64_t(1) << 31) && brows < (int64_t(1) << 31), GDSW_ERR_INVALID_ARG, "GEMM batch too large");
  DevArena loc(s);
  try {
    float* Ac = loc.alloc<float>(arows * W);
    float* Bc = loc.alloc<float>(brows * W);
    SplitTask* dsa = loc.upload(sa, s);
    SplitTask* dsb = loc.upload(sb, s);
    Task* dtasks = loc.upload(tasks, s);
    Tile* dtiles = loc.upload(tiles, s);
    unsigned* derr = loc.alloc<unsigned>(1);
    GDSW_CUDA(cudaMemsetAsync(derr, 0, sizeof(unsigned), s));
    dim3 grid((KpMax + 31) / 32, (Mmax + 31) / 32, unsigned(sa.size()));
    k_tc_split<<<grid, 256, 0, s>>>(dsa, Ac, W, 0);
    check_launch("k_tc_split");
    dim3 gridb((KpMax + 31) / 32, (Nmax + 31) / 32, unsigned(sb.size()));
    k_tc_split<<<gridb, 256, 0, s>>>(dsb, Bc, W, 1);
    check_launch("k_tc_split");
    const CUtensorMap mA = make_map(Ac, arows, W), mB = make_map(Bc, brows, W);
    k_tc_gemm<<<unsigned(tiles.size()), 192, SMEM_BYTES, s>>>(mA, mB, dtasks, dtiles, derr);
    check_launch("k_tc_gemm");
    unsigned herr = 0;
    GDSW_CUDA(cudaMemcpyAsync(&herr, derr, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    GDSW_CUDA(cudaStreamSynchronize(s));
    GDSW_CHECK(herr == 0, GDSW_ERR_TIMEOUT, "tensor-core GEMM: a pipeline wait exceeded its limit");
  } catch (...) {
    loc.free_all();
    throw;
  }
  loc.free_all();
}

}  // namespace gdsw

extern "C" int gdsw_gemm_f32(const gdsw_gemm_task* tasks, int32_t ntasks, int32_t engine) {
  using namespace gdsw;
  if (!tasks || ntasks < 0 || engine < GDSW_GEMM_AUTO || engine > GDSW_GEMM_TENSOR) return GDSW_ERR_INVALID_ARG;
  try {
    std::vector<GemmTaskP> v;
    for (int i = 0; i < ntasks; ++i) {
      const gdsw_gemm_task& t = tasks[i];
      if (!t.a || !t.b || !t.c || t.M < 0 || t.N < 0 || t.K < 0) return GDSW_ERR_INVALID_ARG;
      if (engine == GDSW_GEMM_TENSOR && (t.M < 1 || t.N < 1 || t.K < 1)) return GDSW_ERR_INVALID_ARG;
      v.push_back({t.a, t.b, t.c, t.M, t.N, t.K, t.lda, t.ldb, t.ldc, t.trans_a, t.trans_b, t.alpha, t.beta});
    }
    cudaStream_t s = nullptr;
    if (engine == GDSW_GEMM_TENSOR) {
      run_gemm_tc(v, s);
    } else {
      DevArena tmp(s);
      try {
        run_gemm_engine<float>(tmp, v, s, engine);
        GDSW_CUDA(cudaStreamSynchronize(s));
      } catch (...) {
        tmp.free_all();
        throw;
      }
      tmp.free_all();
    }
    return GDSW_OK;
  } catch (const gdsw::Error& e) {
    return e.code;
  } catch (...) {
    return GDSW_ERR_CUDA;
  }
}

namespace gdsw {
extern bool g_launch_overlap;
}

extern "C" int gdsw_set_launch_overlap(int32_t on) {
  if (on != 0 && on != 1) return GDSW_ERR_INVALID_ARG;
  gdsw::g_launch_overlap = on != 0;
  return GDSW_OK;
}

extern "C" int gdsw_set_gemm_engine(int32_t engine) {
  if (engine < GDSW_GEMM_AUTO || engine > GDSW_GEMM_TENSOR) return GDSW_ERR_INVALID_ARG;
  gdsw::set_gemm_engine(engine);
  return GDSW_OK;
}
