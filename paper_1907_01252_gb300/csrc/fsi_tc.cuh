// 5th-generation tensor-core building blocks for sm_103a (inline PTX):
// tensor-memory allocation, tcgen05.mma of kind::f16 with BF16 operands and an
// FP32 accumulator in tensor memory, completion through an mbarrier, and
// tcgen05.ld of the accumulator.
//
// Operands live in shared memory in the no-swizzle K-major layout: core
// matrices of 8 rows x 16 bytes (8 BF16 values of K), 128 contiguous bytes
// each; core matrix (row group g, K chunk c) starts at (g * kc + c) * 128
// bytes, kc = the K chunks stored per row group. One MMA consumes K = 16,
// i.e. two K-adjacent core matrices (leading-dimension offset 128 B) of every
// row group (stride-dimension offset kc * 128 B).
//
// FP32 values enter as sums of BF16 terms: x = x1 + x2 + x3, x1 the BF16
// rounding of x, x2 of x - x1, x3 of the rest. The product of two such sums
// keeps the six term products whose indices add up to at most four; the
// dropped ones are below FP32 rounding. Each term product is exact in the
// FP32 accumulator's products, so the result has FP32-level accuracy (the
// splitting technique of mixed-precision tensor-core GEMMs).
#pragma once
#include <cstdint>
#include <cuda_bf16.h>

namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (row r, k) of a K-major operand with kc K chunks per row group.
__host__ __device__ __forceinline__ uint32_t kmajor_offset(int r, int k, int kc) {
  return (uint32_t)((((r >> 3) * kc + (k >> 3)) * 8 + (r & 7)) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor: start address, leading (K) and stride
// (row-group) byte offsets, descriptor version 1, no swizzle, base offset 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9 and 10-12 = 1), both K-major, N / 8 in bits 17-22, M / 16 in
// bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Tensor memory: allocated and freed by one whole warp; the base address is
// written to shared memory.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D (tensor memory) = A B^T (+ D when accumulate != 0); issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// The mbarrier receives one arrival when every MMA this thread issued before has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Waits for the completion of the barrier's phase `parity`, at most max_polls
// polls; returns whether it completed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long max_polls) {
  const uint32_t a = smem_u32(bar);
  for (long long i = 0; i < max_polls; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Ordering between ordinary shared-memory stores and the MMA's reads (async
// proxy), and between thread synchronisation and tensor-core operations.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of one tensor-memory lane per thread: warp w
// (w < 4) reads lanes 32 w .. 32 w + 31, thread t lane 32 w + t.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// The BF16 terms of x (NS = 1, 2 or 3 of them).
template <int NS>
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 (&t)[NS]) {
  float r = x;
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    t[i] = __float2bfloat16_rn(r);
    r -= __bfloat162float(t[i]);
  }
}

// The term products (i, j), i + j < NS, of two NS-term splits, in issue order.
template <int NS>
struct SplitPairs {
  static constexpr int count = NS * (NS + 1) / 2;
  __host__ __device__ static constexpr int a(int p) { return NS == 1 ? 0 : (NS == 2 ? (p == 2) : (p < 3 ? 0 : (p < 5 ? 1 : 2))); }
  __host__ __device__ static constexpr int b(int p) { return NS == 1 ? 0 : (NS == 2 ? (p == 1) : (p < 3 ? p : (p < 5 ? p - 3 : 0))); }
};

constexpr long long kMaxPolls = 1ll << 26;   // bounded mbarrier waits

}  // namespace tc

// Tile product D[128][16] = A[128][32] B[16][32]^T of FP32 matrices on the
// tensor cores, each operand entering as NS BF16 terms (the primitive of the
// element contraction, exposed for testing). One CTA of 128 threads; status
// receives 1 if the MMA completion was not seen within the poll limit.
template <int NS>
__global__ void __launch_bounds__(128) k_tc_tile_product(const float* __restrict__ A, const float* __restrict__ B,
                                                        float* __restrict__ D, int* __restrict__ status) {
  // operands in one buffer: NS A terms of 8 KB, NS B terms of 1 KB, then 2 KB of slack
  __shared__ __align__(1024) unsigned char smem[NS * 9216 + 2048];
  unsigned char* sA[NS];
  unsigned char* sB[NS];
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    sA[i] = smem + i * 8192;
    sB[i] = smem + NS * 8192 + i * 1024;
  }
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tc::tmem_alloc(&tmem_base, 32);
  if (tid == 0) tc::mbar_init(&bar, 1);
  for (int e = tid; e < 128 * 32; e += 128) {
    __nv_bfloat16 t[NS];
    tc::split_bf16<NS>(A[e], t);
    const uint32_t o = tc::kmajor_offset(e / 32, e % 32, 4);
#pragma unroll
    for (int i = 0; i < NS; ++i) *reinterpret_cast<__nv_bfloat16*>(sA[i] + o) = t[i];
  }
  for (int e = tid; e < 16 * 32; e += 128) {
    __nv_bfloat16 t[NS];
    tc::split_bf16<NS>(B[e], t);
    const uint32_t o = tc::kmajor_offset(e / 32, e % 32, 4);
#pragma unroll
    for (int i = 0; i < NS; ++i) *reinterpret_cast<__nv_bfloat16*>(sB[i] + o) = t[i];
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  if (tid == 0) {
    constexpr uint32_t idesc = tc::idesc_bf16_f32(128, 16);
    int issued = 0;
    for (int ks = 0; ks < 2; ++ks)
      for (int p = 0; p < tc::SplitPairs<NS>::count; ++p) {
        const uint64_t da = tc::smem_desc(tc::smem_u32(sA[tc::SplitPairs<NS>::a(p)]) + ks * 256, 128, 512);
        const uint64_t db = tc::smem_desc(tc::smem_u32(sB[tc::SplitPairs<NS>::b(p)]) + ks * 256, 128, 512);
        tc::mma_bf16(tmem, da, db, idesc, issued++ > 0);
      }
    tc::mma_commit(&bar);
  }
  __syncwarp();
  bool ok = tc::mbar_wait(&bar, 0, tc::kMaxPolls);
  if (!ok) ok = tc::mbar_wait(&bar, 0, tc::kMaxPolls);   // give the MMAs in flight a second chance
  ok = __syncthreads_and(ok);                            // one outcome for the whole CTA
  if (!ok && tid == 0) atomicExch(status, 1);
  tc::fence_after_sync();
  if (ok) {
    float v[16];
    tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16), v);
#pragma unroll
    for (int n = 0; n < 16; ++n) D[(warp * 32 + lane) * 16 + n] = v[n];
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 32);
}
