// Dense contractions on the fifth-generation tensor cores (tcgen05): C = alpha A B^T with
// float32 inputs split into two bfloat16 terms each (v = hi + lo, hi = bf16(v),
// lo = bf16(v - hi)) and the three products hi hi + hi lo + lo hi accumulated in float32 in
// tensor memory, which keeps about 16 significant bits of every product (the lo lo term and
// the remainders beyond lo are below 2^-16 relative). When B is exact in bfloat16 (the
// network's weights), A may instead be split into three terms, hi + lo + lo2, which carries
// A's full float32 value (terms = 4: three products against B); with both in three terms and
// the six products above 2^-24 relative (terms = 6) the contraction is as accurate as a float32
// one. Used by the warm-start network's 256-wide
// layers (forward, input gradient, weight gradient) and by the column transforms of small grids
// (DST/DCT as a dense 128 x 128 contraction).
//
// One CTA of 128 threads computes a 128 x BN tile of C: K is consumed in chunks of 64; every
// chunk of A and B is staged by the CTA into shared memory in the canonical K-major layout
// (split into hi and lo), one thread issues the MMAs (M = 128, N = BN, K = 16 each), their
// completion arrives on an mbarrier the CTA waits on (bounded), and the four warps read the
// accumulator back from tensor memory (lane = tile row) for the epilogue.
#include <cuda_bf16.h>

#include "kfbi_internal.cuh"
#include "kfbi_tc.cuh"

namespace kfbi {

constexpr int TC_BM = 128, TC_BK = 64, TC_THREADS = 128;
constexpr int TC_WAIT_TRIES = 1 << 20;

template <int BN>
constexpr size_t tc_smem() {
  return 3 * (size_t)TC_BM * TC_BK * 2 + 3 * (size_t)BN * TC_BK * 2 + 64;
}

// stages rows x TC_BK elements of a float32 operand (element (r, k) at p[r ld + k], or p[k ld + r]
// when trans) into the hi and lo tiles (and, with lo2, a third term: v = hi + lo + lo2 to the
// float32 rounding); zero outside rows_valid x k_valid
template <int ROWS>
__device__ __forceinline__ void tc_stage(const float* p, long ld, int trans, int r0, int rows_valid, int k0,
                                         int k_valid, unsigned char* hi, unsigned char* lo, unsigned char* lo2) {
  // sixteen loads in flight per thread before any is used (the staging is L2-latency bound)
  constexpr int PER = ROWS * TC_BK / TC_THREADS, BATCH = 16;
  static_assert(PER % BATCH == 0, "tile rows");
#pragma unroll 1
  for (int b0 = 0; b0 < PER; b0 += BATCH) {
    float v[BATCH];
    int rr[BATCH], kk[BATCH];
#pragma unroll
    for (int u = 0; u < BATCH; ++u) {
      const int e = (int)threadIdx.x + (b0 + u) * TC_THREADS;
      int r, k;
      if (trans) {
        r = e % ROWS;
        k = e / ROWS;
      } else {
        r = e / TC_BK;
        k = e % TC_BK;
      }
      rr[u] = r;
      kk[u] = k;
      const int gr = r0 + r, gk = k0 + k;
      v[u] = (gr < rows_valid && gk < k_valid) ? (trans ? p[(long)gk * ld + gr] : p[(long)gr * ld + gk]) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < BATCH; ++u) {
      const __nv_bfloat16 h = __float2bfloat16_rn(v[u]);
      const float r1 = v[u] - __bfloat162float(h);
      const __nv_bfloat16 l = __float2bfloat16_rn(r1);
      const uint32_t off = tc::kmajor_offset(rr[u], kk[u], TC_BK);
      *(__nv_bfloat16*)(hi + off) = h;
      *(__nv_bfloat16*)(lo + off) = l;
      if (lo2 != nullptr) *(__nv_bfloat16*)(lo2 + off) = __float2bfloat16_rn(r1 - __bfloat162float(l));
    }
  }
}

template <int BN>
__global__ void __launch_bounds__(TC_THREADS) k_tc_gemm(TcGemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  constexpr uint32_t A_BYTES = TC_BM * TC_BK * 2, B_BYTES = BN * TC_BK * 2;
  unsigned char* a_hi = smem_raw;
  unsigned char* a_lo = a_hi + A_BYTES;
  unsigned char* a_lo2 = a_lo + A_BYTES;
  unsigned char* b_hi = a_lo2 + A_BYTES;
  unsigned char* b_lo = b_hi + B_BYTES;
  unsigned char* b_lo2 = b_lo + B_BYTES;
  uint64_t* bar = (uint64_t*)(b_lo2 + B_BYTES);
  uint32_t* tslot = (uint32_t*)(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * BN;
  constexpr uint32_t NCOLS = BN < 32 ? 32 : BN;
  if (warp == 0) tc::tmem_alloc(tslot, NCOLS);
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  constexpr uint32_t IDESC = tc::idesc_bf16_f32(TC_BM, BN);
  constexpr uint32_t LBO = 128, SBO = (TC_BK / 8) * 128;
  const int nchunks = (g.K + TC_BK - 1) / TC_BK;
  int ok = 1, last = 0;
  for (int ch = 0; ch < nchunks && ok; ++ch) {
    const int k0 = ch * TC_BK;
    last = ch;
    tc_stage<TC_BM>(g.A, g.lda, g.transA, m0, g.M, k0, g.K, a_hi, a_lo, g.terms >= 4 ? a_lo2 : nullptr);
    tc_stage<BN>(g.B, g.ldb, g.transB, n0, g.N, k0, g.K, b_hi, b_lo, g.terms == 6 ? b_lo2 : nullptr);
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int s = 0; s < TC_BK / 16; ++s) {
        const uint32_t ko = (uint32_t)s * 256;  // two core matrices along K per MMA
        const uint64_t ah = tc::smem_desc(tc::smem_u32(a_hi) + ko, LBO, SBO);
        const uint64_t al = tc::smem_desc(tc::smem_u32(a_lo) + ko, LBO, SBO);
        const uint64_t bh = tc::smem_desc(tc::smem_u32(b_hi) + ko, LBO, SBO);
        const uint64_t bl = tc::smem_desc(tc::smem_u32(b_lo) + ko, LBO, SBO);
        tc::mma_bf16(tmem, ah, bh, IDESC, (ch > 0 || s > 0) ? 1u : 0u);
        if (g.terms == 3) {
          tc::mma_bf16(tmem, ah, bl, IDESC, 1u);
          tc::mma_bf16(tmem, al, bh, IDESC, 1u);
        } else if (g.terms == 4) {  // B exact in bfloat16: A's three terms against B
          const uint64_t al2 = tc::smem_desc(tc::smem_u32(a_lo2) + ko, LBO, SBO);
          tc::mma_bf16(tmem, al, bh, IDESC, 1u);
          tc::mma_bf16(tmem, al2, bh, IDESC, 1u);
        } else if (g.terms == 6) {  // both in three terms: every product above 2^-24 relative
          const uint64_t al2 = tc::smem_desc(tc::smem_u32(a_lo2) + ko, LBO, SBO);
          const uint64_t bl2 = tc::smem_desc(tc::smem_u32(b_lo2) + ko, LBO, SBO);
          tc::mma_bf16(tmem, ah, bl, IDESC, 1u);
          tc::mma_bf16(tmem, al, bh, IDESC, 1u);
          tc::mma_bf16(tmem, al, bl, IDESC, 1u);
          tc::mma_bf16(tmem, ah, bl2, IDESC, 1u);
          tc::mma_bf16(tmem, al2, bh, IDESC, 1u);
        }
      }
      tc::commit(bar);
    }
    // the chunk's MMAs are done before its tiles are rewritten or the accumulator is read
    const int done = tc::mbar_wait(bar, (uint32_t)(ch & 1), TC_WAIT_TRIES) ? 1 : 0;
    ok = __syncthreads_and(done);
    tc::fence_after_sync();
  }
  if (!ok) {
    if (tid == 0) atomicExch(g.error, 1);
    // the MMAs may still be running: wait once more (bounded) before the memory is released
    tc::mbar_wait(bar, (uint32_t)(last & 1), TC_WAIT_TRIES);
  } else {
    const int r = warp * 32 + lane;  // tile row = tensor-memory lane
    const int gm = m0 + r;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (gm < g.M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int gn = n0 + c0 + j;
          if (gn >= g.N) break;
          float* cp = g.C + (long)gm * g.ldc + gn;
          const float a = g.alpha * v[j];
          if (g.mode == TC_STORE) *cp = a;
          else if (g.mode == TC_ADD) *cp += a;
          else *cp = a / (g.dm[gm] + g.dn[gn] + g.shift);
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, NCOLS);
}

template <int BN>
static kfbi_status tc_launch(const TcGemmArgs& g, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    KFBI_TRY(cudaFuncSetAttribute(k_tc_gemm<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem<BN>()));
    attr = true;
  }
  dim3 grid(cdiv(g.M, TC_BM), cdiv(g.N, BN));
  k_tc_gemm<BN><<<grid, TC_THREADS, tc_smem<BN>(), s>>>(g);
  KFBI_TRY(cudaGetLastError());
  return KFBI_OK;
}

kfbi_status tc_gemm(const TcGemmArgs& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return KFBI_OK;
  const int bn = g.bn > 0 ? g.bn : (g.N > 128 ? 256 : g.N > 64 ? 128 : g.N > 32 ? 64 : 32);
  if (bn >= 256) return tc_launch<256>(g, s);
  if (bn >= 128) return tc_launch<128>(g, s);
  if (bn >= 64) return tc_launch<64>(g, s);
  return tc_launch<32>(g, s);
}

}  // namespace kfbi

extern "C" kfbi_status kfbi_tc_gemm(int M, int N, int K, const float* A, long lda, int transA, const float* B, long ldb,
                                    int transB, float* C, long ldc, int terms, int* error, void* stream) {
  if (M < 1 || N < 1 || K < 1 || A == nullptr || B == nullptr || C == nullptr || error == nullptr) return KFBI_ERR_ARG;
  if ((terms != 1 && terms != 3 && terms != 4 && terms != 6) || lda < 1 || ldb < 1 || ldc < N) return KFBI_ERR_ARG;
  if ((!transA && lda < K) || (transA && lda < M) || (!transB && ldb < K) || (transB && ldb < N)) return KFBI_ERR_ARG;
  kfbi::TcGemmArgs g{};
  g.A = A;
  g.lda = lda;
  g.transA = transA ? 1 : 0;
  g.B = B;
  g.ldb = ldb;
  g.transB = transB ? 1 : 0;
  g.C = C;
  g.ldc = ldc;
  g.M = M;
  g.N = N;
  g.K = K;
  g.alpha = 1.0f;
  g.mode = kfbi::TC_STORE;
  g.terms = terms;
  g.error = error;
  return kfbi::tc_gemm(g, (cudaStream_t)stream);
}
