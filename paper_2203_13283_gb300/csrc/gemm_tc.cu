// Tensor-core contraction for the mixed-precision form: the sampling of the
// skeleton (Eq. 7), the preconditioned right-hand side of Eq. (5) and the
// operator applies of Eq. (6) are dense complex products with the assembled
// Galerkin matrices, carried out here as real products on the 5th-generation
// tensor cores of sm_103a.
//
//   D (M x Nc, FP32) = sum_p  A_{ia[p]} (M x K) * B_{ib[p]} (Nc x K)^T
//
// A and B are bf16 "planes" (split-bf16: x = hi + lo [+ lo2]), K-major (row
// major with K contiguous).  Tiles of A (128 x 64) and B (NT x 64) are staged
// by TMA (128-byte swizzle) into a multi-stage shared-memory ring guarded by
// mbarriers; one thread issues tcgen05.mma (kind::f16, M = 128, N = NT,
// K = 16) accumulating in TMEM; tcgen05.commit releases ring slots; the four
// warps drain TMEM with tcgen05.ld in the epilogue, which applies a complex
// combination (see Epi) and writes FP32 or FP64 output.
//
// Every wait on an mbarrier is bounded; on expiry the kernel records an error
// code in *err, stops issuing work, waits (bounded) for its own copies and
// MMAs, frees TMEM and returns, so the host sees WCS_ERR_TIMEOUT.
#include <cuda.h>

#include <algorithm>

#include "gemm_tc.h"

namespace wcs {

// ----------------------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: gives up after `budget` SM clock cycles, or as soon as any CTA
// of the launch has raised the global error flag.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long budget,
                                          const volatile int* gerr) {
  const long long t0 = clock64();
  for (uint32_t i = 0;; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 255u) == 255u && (clock64() - t0 > budget || *gerr != 0)) return false;
  }
}

// The same wait for warps that share a sub-partition with the MMA-issuing or
// TMA thread: they sleep between polls instead of taking its issue slots.
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t* bar, uint32_t parity, long long budget,
                                                const volatile int* gerr, unsigned ns) {
  const long long t0 = clock64();
  for (uint32_t i = 0;; ++i) {
    if (mbar_try(bar, parity)) return true;
    __nanosleep(ns);
    if ((i & 15u) == 15u && (clock64() - t0 > budget || *gerr != 0)) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ uint64_t sw128_desc(const void* tile) {
  // tcgen05 shared-memory matrix descriptor: K-major, 128-byte swizzle,
  // rows of 128 B, 8-row core groups 1024 B apart (SBO), version 1.
  const uint64_t a = smem_u32(tile);
  uint64_t d = 0;
  d |= (a >> 4) & 0x3FFFull;            // start address
  d |= (uint64_t)1 << 16;               // LBO (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;     // SBO
  d |= (uint64_t)1 << 46;               // descriptor version
  d |= (uint64_t)2 << 61;               // SWIZZLE_128B
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 64 columns of 32 lanes in one load, waited for inside the same statement
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64]) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {"
      "%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
      "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
      "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63"
      "}, [%64];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]),
        "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]),
        "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]),
        "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]),
        "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_st64(uint32_t taddr, const float (&v)[64]) {
  uint32_t r[64];
#pragma unroll
  for (int i = 0; i < 64; ++i) r[i] = __float_as_uint(v[i]);
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x64.b32 [%64], {"
      "%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
      "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
      "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63"
      "};\n"
      "tcgen05.wait::st.sync.aligned;"
      :
      : "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
        "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
        "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31]), "r"(r[32]),
        "r"(r[33]), "r"(r[34]), "r"(r[35]), "r"(r[36]), "r"(r[37]), "r"(r[38]), "r"(r[39]), "r"(r[40]),
        "r"(r[41]), "r"(r[42]), "r"(r[43]), "r"(r[44]), "r"(r[45]), "r"(r[46]), "r"(r[47]), "r"(r[48]),
        "r"(r[49]), "r"(r[50]), "r"(r[51]), "r"(r[52]), "r"(r[53]), "r"(r[54]), "r"(r[55]), "r"(r[56]),
        "r"(r[57]), "r"(r[58]), "r"(r[59]), "r"(r[60]), "r"(r[61]), "r"(r[62]), "r"(r[63]), "r"(taddr)
      : "memory");
}

// ----------------------------------------------------------------------------- kernel
constexpr int TC_BM = 128, TC_BK = 64, TC_THREADS = 128;
constexpr long long WAIT_LIMIT = 4000000000ll;  // SM cycles (~2 s) before a wait is declared stuck

template <int NT, int PA, int PB, int STAGES>
struct TcSmem {
  static constexpr int A_BYTES = TC_BM * TC_BK * 2;   // 16 KB
  static constexpr int B_BYTES = NT * TC_BK * 2;      // 16 or 32 KB
  static constexpr int STAGE_BYTES = PA * A_BYTES + PB * B_BYTES;
  static constexpr int TOTAL = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers, flags*/;
};

template <int NT, int PA, int PB, int STAGES>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
              const __grid_constant__ CUtensorMap mA2, const __grid_constant__ CUtensorMap mB0,
              const __grid_constant__ CUtensorMap mB1, const __grid_constant__ CUtensorMap mB2, TcArgs args) {
  using L = TcSmem<NT, PA, PB, STAGES>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * L::STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tslot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * TC_BM;
  const int n0 = blockIdx.x * NT;
  // split-K: CTA z takes k-blocks [z kper, (z + 1) kper); the host picks kper
  // so that every split is non-empty
  const int nk_all = (args.K + TC_BK - 1) / TC_BK;
  const int kb0 = (args.kper > 0) ? (int)blockIdx.z * args.kper : 0;
  const int nk = (args.kper > 0) ? min(args.kper, nk_all - kb0) : nk_all;

  if (*(volatile int*)args.err != 0) return;  // another CTA already gave up: do nothing
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"((uint32_t)NT));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  const CUtensorMap* mapA[3] = {&mA0, &mA1, &mA2};
  const CUtensorMap* mapB[3] = {&mB0, &mB1, &mB2};
  // instruction descriptor: D f32, A bf16, B bf16, both K-major, N, M
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) |
                         ((uint32_t)(TC_BM >> 4) << 24);

  volatile int* issued = (volatile int*)(tslot + 2);     // k-blocks whose loads were issued
  volatile int* consumed = (volatile int*)(tslot + 3);   // k-blocks the MMA thread waited for
  if (threadIdx.x == 0) { *issued = 0; *consumed = 0; }
  __syncthreads();
  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      if (kb >= STAGES) {
        if (!mbar_wait(&empty[s], ((kb / STAGES) + 1) & 1, WAIT_LIMIT, args.err)) { *abort_flag = 11; break; }
      }
      if (*abort_flag) break;
      uint8_t* st = smem + s * L::STAGE_BYTES;
      mbar_expect_tx(&full[s], L::STAGE_BYTES);
      const int k0 = (kb0 + kb) * TC_BK;
#pragma unroll
      for (int p = 0; p < PA; ++p) tma_load_2d(st + p * L::A_BYTES, mapA[p], &full[s], k0, m0);
#pragma unroll
      for (int p = 0; p < PB; ++p) tma_load_2d(st + PA * L::A_BYTES + p * L::B_BYTES, mapB[p], &full[s], k0, n0);
      *issued = kb + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      if (!mbar_wait(&full[s], (kb / STAGES) & 1, WAIT_LIMIT, args.err)) { *abort_flag = 12; break; }
      *consumed = kb + 1;
      if (*abort_flag) break;
      tc_fence_after();
      uint8_t* st = smem + s * L::STAGE_BYTES;
      for (int p = 0; p < args.nprod; ++p) {
        const uint8_t* ta = st + args.ia[p] * L::A_BYTES;
        const uint8_t* tb = st + PA * L::A_BYTES + args.ib[p] * L::B_BYTES;
        const uint64_t da = sw128_desc(ta), db = sw128_desc(tb);
#pragma unroll
        for (int kk = 0; kk < TC_BK / 16; ++kk) {
          // advance 16 bf16 = 32 bytes along K inside the swizzle atom
          mma_bf16(tmem, da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), idesc,
                   (kb > 0 || p > 0 || kk > 0) ? 1u : 0u);
        }
      }
      mma_commit(&empty[s]);
    }
    mma_commit(done);   // arrives once every MMA issued above has completed
  }
  __syncwarp();
  // ---------------- epilogue: all four warps
  bool got = mbar_wait(done, 0, WAIT_LIMIT, args.err);
  const bool waited = __all_sync(0xffffffffu, got);
  got = waited && (__shfl_sync(0xffffffffu, *abort_flag, 0) == 0);
  tc_fence_after();
  if (!got) {
    if (!waited && lane == 0) atomicCAS((int*)abort_flag, 0, 13);
    __syncwarp();
    if (threadIdx.x == 0) {
      const int zero_flag = 0;
      atomicExch(args.err, 1000 * (*abort_flag) + (int)(blockIdx.x % 1000));
      // let the loads already in flight land before the CTA's shared memory goes away
      for (int kb = *consumed; kb < *issued; ++kb)
        (void)mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1, WAIT_LIMIT, &zero_flag);
    }
  } else {
    const int row = m0 + warp * 32 + lane;   // TMEM lane = tile row
#pragma unroll 1
    for (int c0 = 0; c0 < NT; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (args.ws) {
        // split-K partial, column-major [split][Nc][M]: a warp writes 32 consecutive rows per column
        if (row < args.M) {
          float* w = args.ws + (int64_t)blockIdx.z * args.Nc * args.M + row;
#pragma unroll
          for (int i = 0; i < 32; ++i)
            if (n0 + c0 + i < args.Nc) w[(int64_t)(n0 + c0 + i) * args.M] = v[i];
        }
      } else {
        epilogue_store(args, row, n0 + c0, v);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)NT));
  }
}

// ----------------------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// bf16 matrix rows x cols (K = cols contiguous), leading dimension ld elements
static int make_map(CUtensorMap* m, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) { set_error("cuTensorMapEncodeTiled unavailable"); return 3; }
  if (((uintptr_t)base & 15) || ((ld * 2) & 15)) { set_error("tensor map: base or pitch not 16-byte aligned"); return 1; }
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) { set_error("cuTensorMapEncodeTiled failed"); return 3; }
  return 0;
}

template <int NT, int PA, int PB, int STAGES>
static int launch_tc(const TcOperand& A, const TcOperand& B, TcArgs& args, cudaStream_t s) {
  using L = TcSmem<NT, PA, PB, STAGES>;
  CUtensorMap ma[3], mb[3];
  std::memset(ma, 0, sizeof(ma));
  std::memset(mb, 0, sizeof(mb));
  for (int p = 0; p < PA; ++p) TRY_TC(make_map(&ma[p], A.plane[p], args.M, args.K, A.ld, TC_BM));
  for (int p = 0; p < PB; ++p) TRY_TC(make_map(&mb[p], B.plane[p], args.Nc, args.K, B.ld, NT));
  for (int p = PA; p < 3; ++p) ma[p] = ma[0];
  for (int p = PB; p < 3; ++p) mb[p] = mb[0];
  auto kern = k_gemm_tc<NT, PA, PB, STAGES>;
  static DeviceOnce attr;   // one instance per template instantiation
  if (attr.need()) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::TOTAL);
    if (e != cudaSuccess) { set_error(std::string("gemm_tc: shared-memory opt-in: ") + cudaGetErrorString(e)); return 3; }
    attr.done();
  }
  const int nk = (args.K + TC_BK - 1) / TC_BK;
  const int splits = (args.kper > 0) ? (nk + args.kper - 1) / args.kper : 1;
  dim3 grid((unsigned)((args.Nc + NT - 1) / NT), (unsigned)((args.M + TC_BM - 1) / TC_BM), (unsigned)splits);
  kern<<<grid, TC_THREADS, L::TOTAL, s>>>(ma[0], ma[1], ma[2], mb[0], mb[1], mb[2], args);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error(std::string("gemm_tc launch: ") + cudaGetErrorString(e)); return 3; }
  return 0;
}

// Sum of the split-K partials in a fixed order (FP64) and the epilogue.
__global__ void k_splitk_reduce(TcArgs a, int splits) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t plane = (int64_t)a.Nc * a.M;
  if (a.epi == EPI_RAW_F64) {
    if (t >= plane) return;
    const int row = (int)(t % a.M), col = (int)(t / a.M);
    double sum = 0.0;
    for (int z = 0; z < splits; ++z) sum += (double)a.ws[z * plane + t];
    double* o = (double*)a.out + (int64_t)row * a.ldo + col;
    *o = a.alpha.x * sum + ((a.beta.x == 0.0) ? 0.0 : a.beta.x * (*o));
    return;
  }
  const int ncols = a.Nc / 2;
  if (t >= (int64_t)a.M * ncols) return;
  const int row = (int)(t % a.M), j = (int)(t / a.M);
  const float* w = a.ws + (int64_t)(2 * j) * a.M + row;
  double re = 0.0, im = 0.0;
  for (int z = 0; z < splits; ++z) {
    re += (double)w[z * plane];
    im += (double)w[z * plane + a.M];
  }
  zd p = mkz(re, a.conj_out ? -im : im);
  p = a.alpha * p;
  zd* o = (zd*)a.out + (int64_t)j * a.ldo + row;
  if (!(a.beta.x == 0.0 && a.beta.y == 0.0)) p += a.beta * (*o);
  *o = p;
}


// ----------------------------------------------------------------------------- accurate variant
// The tensor-core accumulator truncates: its relative error grows with the
// number of accumulation steps (measured ~3e-8 per step).  This variant keeps
// each K = 16 step's result in its own TMEM buffer (two buffers, ping-pong),
// and eight drain warps move it into FP32 registers before the next use, so no
// TMEM sum spans more than one step.  Register sums are two-level (an inner
// sum over 64 steps folded into an outer sum), which keeps the FP32 rounding
// of ~K/16 additions near 1e-7 at a quarter of the cost of compensated
// summation.  Tile 128 x 128; warps 0-7 drain (warp w: TMEM lanes 32 (w % 4),
// columns 64 (w / 4)), warp 8 loads (TMA), warp 9 issues the MMAs.  The drain
// is bound by the latency of the TMEM load, so each warp moves its 64 columns
// in one load and keeps only the inner sums in registers; the outer sums live
// in the last 128 TMEM columns, after three step buffers (384 columns).
constexpr int ACC_NT = 128, ACC_THREADS = 320, ACC_FOLD = 64, ACC_NBUF = 3;
constexpr int ACC_OUTER = ACC_NBUF * ACC_NT;   // first TMEM column of the outer sums

template <int PA, int PB, int STAGES>
struct AccSmem {
  static constexpr int A_BYTES = TC_BM * TC_BK * 2;        // 16 KB
  static constexpr int B_BYTES = ACC_NT * TC_BK * 2;       // 16 KB
  static constexpr int STAGE_BYTES = PA * A_BYTES + PB * B_BYTES;
  static constexpr int TOTAL = STAGES * STAGE_BYTES + 1024 + 256;
};

template <int PA, int PB, int STAGES>
__global__ void __launch_bounds__(ACC_THREADS, 1)
    k_gemm_tc_acc(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
                  const __grid_constant__ CUtensorMap mA2, const __grid_constant__ CUtensorMap mB0,
                  const __grid_constant__ CUtensorMap mB1, const __grid_constant__ CUtensorMap mB2, TcArgs args) {
  using L = AccSmem<PA, PB, STAGES>;
  extern __shared__ uint8_t smem_raw[];
  if (*(volatile int*)args.err != 0) return;
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * L::STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;      // [ACC_NBUF] MMA -> drain
  uint64_t* tempty = tfull + ACC_NBUF;   // [ACC_NBUF] drain -> MMA
  uint32_t* tslot = (uint32_t*)(tempty + ACC_NBUF);
  volatile int* abort_flag = (volatile int*)(tslot + 1);
  volatile int* issued = (volatile int*)(tslot + 2);
  volatile int* consumed = (volatile int*)(tslot + 3);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * TC_BM;
  const int n0 = blockIdx.x * ACC_NT;
  const int nk = (args.K + TC_BK - 1) / TC_BK;
  const int nsteps = nk * (TC_BK / 16);
  // accumulation groups: `drain` consecutive K = 16 steps share one TMEM
  // buffer before it is drained (1: every step)
  const int drain = args.drain > 1 ? args.drain : 1;
  const int ngroups = (nsteps + drain - 1) / drain;

  if (threadIdx.x == 0) {
    for (int q = 0; q < STAGES; ++q) { mbar_init(&full[q], 1); mbar_init(&empty[q], 1); }
    for (int q = 0; q < ACC_NBUF; ++q) { mbar_init(&tfull[q], 1); mbar_init(&tempty[q], 8); }
    *abort_flag = 0;
    *issued = 0;
    *consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(512u));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const CUtensorMap* mapA[3] = {&mA0, &mA1, &mA2};
  const CUtensorMap* mapB[3] = {&mB0, &mB1, &mB2};
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(ACC_NT >> 3) << 17) |
                         ((uint32_t)(TC_BM >> 4) << 24);

  float inner[64];
#pragma unroll
  for (int i = 0; i < 64; ++i) inner[i] = 0.f;

  if (warp == 8) {
    if (lane == 0) {
      for (int kb = 0; kb < nk; ++kb) {
        const int st = kb % STAGES;
        if (kb >= STAGES) {
          if (!mbar_wait(&empty[st], ((kb / STAGES) + 1) & 1, WAIT_LIMIT, args.err)) { *abort_flag = 21; break; }
        }
        if (*abort_flag) break;
        uint8_t* sp = smem + st * L::STAGE_BYTES;
        mbar_expect_tx(&full[st], L::STAGE_BYTES);
        const int k0 = kb * TC_BK;
#pragma unroll
        for (int p = 0; p < PA; ++p) tma_load_2d(sp + p * L::A_BYTES, mapA[p], &full[st], k0, m0);
#pragma unroll
        for (int p = 0; p < PB; ++p) tma_load_2d(sp + PA * L::A_BYTES + p * L::B_BYTES, mapB[p], &full[st], k0, n0);
        *issued = kb + 1;
      }
    }
  } else if (warp == 9) {
    if (lane == 0) {
      // products of order < planes, smallest first (the order of tc_products,
      // checked on the host); descriptors are formed once per stage and the
      // group/buffer counters advance without divisions, so the issuing thread
      // keeps ahead of the tensor core
      constexpr int NP = (PA == 3) ? 6 : 3;
      constexpr int IA[6] = {PA == 3 ? 2 : 1, PA == 3 ? 1 : 0, 0, 1, 0, 0};
      constexpr int IB[6] = {0, 1, PA == 3 ? 2 : 0, 0, 1, 0};
      int b = 0, ingroup = 0, q = 0;
      bool ok = true;
      for (int kb = 0; kb < nk && ok; ++kb) {
        const int st = kb % STAGES;
        if (!mbar_wait(&full[st], (kb / STAGES) & 1, WAIT_LIMIT, args.err)) { *abort_flag = 22; break; }
        *consumed = kb + 1;
        if (*abort_flag) break;
        tc_fence_after();
        const uint8_t* sp = smem + st * L::STAGE_BYTES;
        uint64_t da[NP], db[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          da[p] = sw128_desc(sp + IA[p] * L::A_BYTES);
          db[p] = sw128_desc(sp + PA * L::A_BYTES + IB[p] * L::B_BYTES);
        }
        if (drain == TC_BK / 16) {
          // one group per stage, issued product-major: every step's small
          // plane products enter the fresh accumulator before any large one,
          // so the truncating accumulator cuts them at their own scale, not
          // at the scale of the leading product
          if (q >= ACC_NBUF) {
            if (!mbar_wait(&tempty[b], ((q / ACC_NBUF) - 1) & 1, WAIT_LIMIT, args.err)) {
              *abort_flag = 25;
              mma_commit(&empty[st]);
              break;
            }
            tc_fence_after();
          }
          const uint32_t dt = tmem + (uint32_t)(b * ACC_NT);
#pragma unroll
          for (int p = 0; p < NP; ++p)
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk)
              mma_bf16(dt, da[p] + (uint64_t)(2 * kk), db[p] + (uint64_t)(2 * kk), idesc,
                       (p == 0 && kk == 0) ? 0u : 1u);
          mma_commit(&tfull[b]);
          ++q;
          b = (b == ACC_NBUF - 1) ? 0 : b + 1;
          mma_commit(&empty[st]);
          continue;
        }
#pragma unroll
        for (int kk = 0; kk < TC_BK / 16; ++kk) {
          if (ingroup == 0 && q >= ACC_NBUF) {
            if (!mbar_wait(&tempty[b], ((q / ACC_NBUF) - 1) & 1, WAIT_LIMIT, args.err)) {
              *abort_flag = 25; ok = false; break;
            }
            tc_fence_after();
          }
          const uint32_t dt = tmem + (uint32_t)(b * ACC_NT);
#pragma unroll
          for (int p = 0; p < NP; ++p)
            mma_bf16(dt, da[p] + (uint64_t)(2 * kk), db[p] + (uint64_t)(2 * kk), idesc,
                     (ingroup == 0 && p == 0) ? 0u : 1u);
          ++ingroup;
          if (ingroup == drain || (kb == nk - 1 && kk == TC_BK / 16 - 1)) {
            mma_commit(&tfull[b]);
            ingroup = 0;
            ++q;
            b = (b == ACC_NBUF - 1) ? 0 : b + 1;
          }
        }
        mma_commit(&empty[st]);
      }
    }
  } else {
    // drain warps
    const int lanebase = 32 * (warp & 3), colhalf = 64 * (warp >> 2);
    const uint32_t touter = tmem + ((uint32_t)lanebase << 16) + (uint32_t)(ACC_OUTER + colhalf);
    float v[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = 0.f;
    tmem_st64(touter, v);
    for (int g = 0; g < ngroups; ++g) {
      const int b = g % ACC_NBUF;
      bool got = (drain > 1) ? mbar_wait_sleep(&tfull[b], (g / ACC_NBUF) & 1, WAIT_LIMIT, args.err, 256u)
                             : mbar_wait(&tfull[b], (g / ACC_NBUF) & 1, WAIT_LIMIT, args.err);
      got = __all_sync(0xffffffffu, got) && (__shfl_sync(0xffffffffu, *abort_flag, 0) == 0);
      if (!got) { if (lane == 0) atomicCAS((int*)abort_flag, 0, 24); break; }
      tc_fence_after();
      tmem_ld64(tmem + ((uint32_t)lanebase << 16) + (uint32_t)(b * ACC_NT + colhalf), v);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[b])) : "memory");
#pragma unroll
      for (int i = 0; i < 64; ++i) inner[i] += v[i];
      if ((g % ACC_FOLD) == ACC_FOLD - 1) {
        tmem_ld64(touter, v);
#pragma unroll
        for (int i = 0; i < 64; ++i) { v[i] += inner[i]; inner[i] = 0.f; }
        tmem_st64(touter, v);
      }
    }
  }
  __syncthreads();
  const bool ok = (*abort_flag == 0);
  if (!ok) {
    if (threadIdx.x == 0) {
      const int zero_flag = 0;
      atomicExch(args.err, 1000 * (*abort_flag) + (int)(blockIdx.x % 1000));
      for (int kb = *consumed; kb < *issued; ++kb)
        (void)mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1, WAIT_LIMIT, &zero_flag);
    }
  } else if (warp < 8) {
    const int lanebase = 32 * (warp & 3), colhalf = 64 * (warp >> 2);
    float v[64], out[32];
    tmem_ld64(tmem + ((uint32_t)lanebase << 16) + (uint32_t)(ACC_OUTER + colhalf), v);
#pragma unroll
    for (int i = 0; i < 32; ++i) out[i] = v[i] + inner[i];
    epilogue_store(args, m0 + lanebase + lane, n0 + colhalf, out);
#pragma unroll
    for (int i = 0; i < 32; ++i) out[i] = v[32 + i] + inner[32 + i];
    epilogue_store(args, m0 + lanebase + lane, n0 + colhalf + 32, out);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u));
  }
}

template <int PA, int PB, int STAGES>
static int launch_tc_acc(const TcOperand& A, const TcOperand& B, TcArgs& args, cudaStream_t s) {
  using L = AccSmem<PA, PB, STAGES>;
  CUtensorMap ma[3], mb[3];
  std::memset(ma, 0, sizeof(ma));
  std::memset(mb, 0, sizeof(mb));
  for (int p = 0; p < PA; ++p) TRY_TC(make_map(&ma[p], A.plane[p], args.M, args.K, A.ld, TC_BM));
  for (int p = 0; p < PB; ++p) TRY_TC(make_map(&mb[p], B.plane[p], args.Nc, args.K, B.ld, ACC_NT));
  for (int p = PA; p < 3; ++p) ma[p] = ma[0];
  for (int p = PB; p < 3; ++p) mb[p] = mb[0];
  auto kern = k_gemm_tc_acc<PA, PB, STAGES>;
  static DeviceOnce attr;   // one instance per template instantiation
  if (attr.need()) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::TOTAL);
    if (e != cudaSuccess) { set_error(std::string("gemm_tc: shared-memory opt-in: ") + cudaGetErrorString(e)); return 3; }
    attr.done();
  }
  dim3 grid((unsigned)((args.Nc + ACC_NT - 1) / ACC_NT), (unsigned)((args.M + TC_BM - 1) / TC_BM));
  kern<<<grid, ACC_THREADS, L::TOTAL, s>>>(ma[0], ma[1], ma[2], mb[0], mb[1], mb[2], args);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error(std::string("gemm_tc_acc launch: ") + cudaGetErrorString(e)); return 3; }
  return 0;
}

// ----------------------------------------------------------------------------- periodic drain, wide tile
// The periodic mode (two planes, three products, accumulator drained every
// `drain` K = 16 steps) on 128 x 256 tiles.  With 128 x 128 tiles its three
// products per 64 KB stage (96 flop per staged byte) starved the tensor pipe
// on the L2-to-shared-memory feed; 128 x 256 tiles carry 131 flop per byte,
// like the one-accumulator kernel.  Two TMEM accumulators of 256 columns fill
// the 512 TMEM columns, so the drained sums stay in registers: warp w of the
// eight drain warps owns TMEM lanes 32 (w % 4) and columns 128 (w / 4), 128
// FP32 sums per thread.  A single level of sums suffices: K / (16 drain)
// additions (64 at K = 65536) round far below this mode's ~1e-5.
constexpr int PER_NT = 256, PER_THREADS = 320;

template <int STAGES>
struct PerSmem {
  static constexpr int A_BYTES = TC_BM * TC_BK * 2;        // 16 KB
  static constexpr int B_BYTES = PER_NT * TC_BK * 2;       // 32 KB
  static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr int TOTAL = STAGES * STAGE_BYTES + 1024 + 256;
};

template <int STAGES>
__global__ void __launch_bounds__(PER_THREADS, 1)
    k_gemm_tc_per(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
                  const __grid_constant__ CUtensorMap mB0, const __grid_constant__ CUtensorMap mB1, TcArgs args) {
  using L = PerSmem<STAGES>;
  extern __shared__ uint8_t smem_raw[];
  if (*(volatile int*)args.err != 0) return;
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * L::STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;      // [2] MMA -> drain
  uint64_t* tempty = tfull + 2;          // [2] drain -> MMA
  uint32_t* tslot = (uint32_t*)(tempty + 2);
  volatile int* abort_flag = (volatile int*)(tslot + 1);
  volatile int* issued = (volatile int*)(tslot + 2);
  volatile int* consumed = (volatile int*)(tslot + 3);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * TC_BM;
  const int n0 = blockIdx.x * PER_NT;
  const int nk = (args.K + TC_BK - 1) / TC_BK;
  const int nsteps = nk * (TC_BK / 16);
  const int drain = args.drain > 1 ? args.drain : 1;
  const int ngroups = (nsteps + drain - 1) / drain;

  if (threadIdx.x == 0) {
    for (int q = 0; q < STAGES; ++q) { mbar_init(&full[q], 1); mbar_init(&empty[q], 1); }
    for (int q = 0; q < 2; ++q) { mbar_init(&tfull[q], 1); mbar_init(&tempty[q], 8); }
    *abort_flag = 0;
    *issued = 0;
    *consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(512u));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(PER_NT >> 3) << 17) |
                         ((uint32_t)(TC_BM >> 4) << 24);

  float sum[128];
#pragma unroll
  for (int i = 0; i < 128; ++i) sum[i] = 0.f;

  if (warp == 8) {
    if (lane == 0) {
      for (int kb = 0; kb < nk; ++kb) {
        const int st = kb % STAGES;
        if (kb >= STAGES) {
          if (!mbar_wait(&empty[st], ((kb / STAGES) + 1) & 1, WAIT_LIMIT, args.err)) { *abort_flag = 31; break; }
        }
        if (*abort_flag) break;
        uint8_t* sp = smem + st * L::STAGE_BYTES;
        mbar_expect_tx(&full[st], L::STAGE_BYTES);
        const int k0 = kb * TC_BK;
        tma_load_2d(sp, &mA0, &full[st], k0, m0);
        tma_load_2d(sp + L::A_BYTES, &mA1, &full[st], k0, m0);
        tma_load_2d(sp + 2 * L::A_BYTES, &mB0, &full[st], k0, n0);
        tma_load_2d(sp + 2 * L::A_BYTES + L::B_BYTES, &mB1, &full[st], k0, n0);
        *issued = kb + 1;
      }
    }
  } else if (warp == 9) {
    if (lane == 0) {
      // products of order < 2, smallest first: A1 B0, A0 B1, A0 B0
      constexpr int IA[3] = {1, 0, 0};
      constexpr int IB[3] = {0, 1, 0};
      int b = 0, ingroup = 0, q = 0;
      bool ok = true;
      for (int kb = 0; kb < nk && ok; ++kb) {
        const int st = kb % STAGES;
        if (!mbar_wait(&full[st], (kb / STAGES) & 1, WAIT_LIMIT, args.err)) { *abort_flag = 32; break; }
        *consumed = kb + 1;
        if (*abort_flag) break;
        tc_fence_after();
        const uint8_t* sp = smem + st * L::STAGE_BYTES;
        uint64_t da[3], db[3];
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          da[p] = sw128_desc(sp + IA[p] * L::A_BYTES);
          db[p] = sw128_desc(sp + 2 * L::A_BYTES + IB[p] * L::B_BYTES);
        }
#pragma unroll
        for (int kk = 0; kk < TC_BK / 16; ++kk) {
          if (ingroup == 0 && q >= 2) {
            if (!mbar_wait(&tempty[b], ((q / 2) - 1) & 1, WAIT_LIMIT, args.err)) {
              *abort_flag = 35; ok = false; break;
            }
            tc_fence_after();
          }
          const uint32_t dt = tmem + (uint32_t)(b * PER_NT);
#pragma unroll
          for (int p = 0; p < 3; ++p)
            mma_bf16(dt, da[p] + (uint64_t)(2 * kk), db[p] + (uint64_t)(2 * kk), idesc,
                     (ingroup == 0 && p == 0) ? 0u : 1u);
          ++ingroup;
          if (ingroup == drain || (kb == nk - 1 && kk == TC_BK / 16 - 1)) {
            mma_commit(&tfull[b]);
            ingroup = 0;
            ++q;
            b ^= 1;
          }
        }
        mma_commit(&empty[st]);
      }
    }
  } else {
    // drain warps: sums of their 32 lanes x 128 columns in registers
    const int lanebase = 32 * (warp & 3), colbase = 128 * (warp >> 2);
    for (int g = 0; g < ngroups; ++g) {
      const int b = g & 1;
      bool got = mbar_wait_sleep(&tfull[b], (g >> 1) & 1, WAIT_LIMIT, args.err, 256u);
      got = __all_sync(0xffffffffu, got) && (__shfl_sync(0xffffffffu, *abort_flag, 0) == 0);
      if (!got) { if (lane == 0) atomicCAS((int*)abort_flag, 0, 34); break; }
      tc_fence_after();
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)lanebase << 16) + (uint32_t)(b * PER_NT + colbase + 32 * c4), v);
#pragma unroll
        for (int i = 0; i < 32; ++i) sum[32 * c4 + i] += v[i];
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[b])) : "memory");
    }
  }
  __syncthreads();
  const bool ok = (*abort_flag == 0);
  if (!ok) {
    if (threadIdx.x == 0) {
      const int zero_flag = 0;
      atomicExch(args.err, 1000 * (*abort_flag) + (int)(blockIdx.x % 1000));
      for (int kb = *consumed; kb < *issued; ++kb)
        (void)mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1, WAIT_LIMIT, &zero_flag);
    }
  } else if (warp < 8) {
    const int lanebase = 32 * (warp & 3), colbase = 128 * (warp >> 2);
#pragma unroll
    for (int c4 = 0; c4 < 4; ++c4) {
      float out[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) out[i] = sum[32 * c4 + i];
      epilogue_store(args, m0 + lanebase + lane, n0 + colbase + 32 * c4, out);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u));
  }
}

template <int STAGES>
static int launch_tc_per(const TcOperand& A, const TcOperand& B, TcArgs& args, cudaStream_t s) {
  using L = PerSmem<STAGES>;
  CUtensorMap ma[2], mb[2];
  std::memset(ma, 0, sizeof(ma));
  std::memset(mb, 0, sizeof(mb));
  for (int p = 0; p < 2; ++p) TRY_TC(make_map(&ma[p], A.plane[p], args.M, args.K, A.ld, TC_BM));
  for (int p = 0; p < 2; ++p) TRY_TC(make_map(&mb[p], B.plane[p], args.Nc, args.K, B.ld, PER_NT));
  auto kern = k_gemm_tc_per<STAGES>;
  static DeviceOnce attr;
  if (attr.need()) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::TOTAL);
    if (e != cudaSuccess) { set_error(std::string("gemm_tc: shared-memory opt-in: ") + cudaGetErrorString(e)); return 3; }
    attr.done();
  }
  dim3 grid((unsigned)((args.Nc + PER_NT - 1) / PER_NT), (unsigned)((args.M + TC_BM - 1) / TC_BM));
  kern<<<grid, PER_THREADS, L::TOTAL, s>>>(ma[0], ma[1], mb[0], mb[1], args);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error(std::string("gemm_tc_per launch: ") + cudaGetErrorString(e)); return 3; }
  return 0;
}

int gemm_tc_accurate(const TcOperand& A, const TcOperand& B, TcArgs args, cudaStream_t s) {
  if (args.M <= 0 || args.Nc <= 0 || args.K <= 0) return 0;
  if (args.nprod < 1 || args.nprod > 6) { set_error("gemm_tc: 1..6 products"); return 1; }
  for (int p = 0; p < args.nprod; ++p)
    if (args.ia[p] >= A.planes || args.ib[p] >= B.planes) { set_error("gemm_tc: plane index"); return 1; }
  if ((args.M + TC_BM - 1) / TC_BM > 65535) { set_error("gemm_tc: M too large"); return 1; }
  {
    // the kernel issues the full product list of tc_products for its plane count
    TcArgs ref;
    tc_products(A.planes, ref);
    bool same = (A.planes == B.planes) && (args.nprod == ref.nprod);
    for (int p = 0; same && p < ref.nprod; ++p) same = (args.ia[p] == ref.ia[p] && args.ib[p] == ref.ib[p]);
    if (!same) { set_error("gemm_tc_accurate: needs the full product list of tc_products"); return 1; }
  }
  if (A.planes == 3 && B.planes == 3) return launch_tc_acc<3, 3, 2>(A, B, args, s);
  // two planes drained every 16 or more steps on a grid of more than one
  // column tile: the wide-tile kernel
  if (A.planes == 2 && B.planes == 2 && args.drain >= 16 && args.Nc > 128) return launch_tc_per<2>(A, B, args, s);
  if (A.planes == 2 && B.planes == 2) return launch_tc_acc<2, 2, 3>(A, B, args, s);
  set_error("gemm_tc_accurate: plane combination not built");
  return 1;
}

int gemm_tc_split_plan(int M, int Nc, int K, int planesA, int planesB, int epi, int64_t* ws_elems) {
  *ws_elems = 0;
  if (M <= 0 || Nc <= 0 || K <= 0) return 0;
  if (!(epi == EPI_RAW_F64 || (epi == EPI_CPLX_F64 && (Nc % 2) == 0))) return 0;
  const int NT = ((planesA == 3 && planesB == 3) || Nc <= 128) ? 128 : 256;
  const int nk = (K + TC_BK - 1) / TC_BK;
  const int64_t ctas = (int64_t)((Nc + NT - 1) / NT) * ((M + TC_BM - 1) / TC_BM);
  if (ctas >= 152 || nk < 8) return 0;
  int64_t want = (2 * 152 + ctas - 1) / ctas;
  want = std::min<int64_t>(want, nk / 4);
  // at most 64 MB of partials
  want = std::min<int64_t>(want, ((int64_t)1 << 24) / ((int64_t)Nc * M));
  if (want <= 1) return 0;
  const int kper = (int)((nk + want - 1) / want);
  const int splits = (nk + kper - 1) / kper;   // <= want, every split non-empty
  *ws_elems = (int64_t)splits * Nc * M;
  return kper;
}

int gemm_tc(const TcOperand& A, const TcOperand& B, TcArgs args, cudaStream_t s) {
  if (args.M <= 0 || args.Nc <= 0 || args.K <= 0) return 0;
  if (args.nprod < 1 || args.nprod > 6) { set_error("gemm_tc: 1..6 products"); return 1; }
  if (A.planes < 1 || A.planes > 3 || B.planes < 1 || B.planes > 3) { set_error("gemm_tc: 1..3 planes"); return 1; }
  for (int p = 0; p < args.nprod; ++p)
    if (args.ia[p] >= A.planes || args.ib[p] >= B.planes) { set_error("gemm_tc: plane index"); return 1; }
  if ((args.M + TC_BM - 1) / TC_BM > 65535) { set_error("gemm_tc: M too large"); return 1; }
  const int key = A.planes * 10 + B.planes;
  const int NT = (key == 33 || args.Nc <= 128) ? 128 : 256;
  // split-K when the output tiles cannot fill the GPU (tall-K products such
  // as Q^H Y with few rows); needs the caller's FP32 workspace
  float* ws = args.ws;
  args.ws = nullptr;
  args.kper = 0;
  int splits = 1;
  if (ws && args.force_kper > 0) {
    const int nk = (args.K + TC_BK - 1) / TC_BK;
    const int kper = args.force_kper;
    splits = (nk + kper - 1) / kper;
    if ((int64_t)splits * args.Nc * args.M > args.ws_elems) { set_error("gemm_tc: split-K workspace too small"); return 1; }
    args.kper = kper;
    args.ws = ws;
  } else if (ws) {
    int64_t need = 0;
    const int kper = gemm_tc_split_plan(args.M, args.Nc, args.K, A.planes, B.planes, args.epi, &need);
    if (kper > 0 && need <= args.ws_elems) {
      args.kper = kper;
      args.ws = ws;
      const int nk = (args.K + TC_BK - 1) / TC_BK;
      splits = (nk + kper - 1) / kper;
    }
  }
  int r = 0;
  switch (key) {
    case 11: r = (NT == 128) ? launch_tc<128, 1, 1, 4>(A, B, args, s) : launch_tc<256, 1, 1, 4>(A, B, args, s); break;
    case 22: r = (NT == 128) ? launch_tc<128, 2, 2, 3>(A, B, args, s) : launch_tc<256, 2, 2, 2>(A, B, args, s); break;
    case 33: r = launch_tc<128, 3, 3, 2>(A, B, args, s); break;
    default: set_error("gemm_tc: plane combination not built"); return 1;
  }
  if (r || args.no_reduce || splits == 1) return r;
  const int64_t n = (int64_t)args.M * ((args.epi == EPI_RAW_F64) ? args.Nc : args.Nc / 2);
  k_splitk_reduce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(args, splits);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error(std::string("split-K reduce: ") + cudaGetErrorString(e)); return 3; }
  return 0;
}

}  // namespace wcs
