// tc_gemm.cuh -- a 128 x 128 TF32 tensor-core tile for sm_103a (5th-generation tensor cores):
//   acc[128 x 128] = A[128 x K] * B[128 x K]^T   (FP32 accumulation in tensor memory)
// Operands are FP32 rows with K contiguous (K-major), staged into shared memory by cp.async in the
// no-swizzle core-matrix layout (8 rows x 16 bytes per core matrix), consumed by tcgen05.mma kind::tf32 issued
// by one thread, accumulated in TMEM (128 lanes x 128 columns) and read back with tcgen05.ld.
// K is processed in chunks of 32 (four K=8 instructions per chunk) through a two-stage pipeline; the mbarrier
// completion of a chunk's instructions frees its stage. Every wait is bounded; a wait that runs out sets an
// error flag (GP_ERR_TIMEOUT) and the tile is abandoned after the outstanding work drains, so nothing spins
// forever.
#pragma once
#include <stdint.h>

namespace tcg {

constexpr int TM = 128;                  // rows of A / lanes of the accumulator
constexpr int TN = 128;                  // rows of B / accumulator columns
constexpr int KC = 32;                   // K elements per chunk (128 bytes of FP32)
constexpr int STAGE_BYTES = TM * KC * 4; // 16 KB per operand per stage
constexpr int SMEM_BYTES = 4 * STAGE_BYTES + 1024;   // A0 A1 B0 B1 + barriers/slack
constexpr uint32_t WAIT_LIMIT = 1u << 26;             // bounded mbarrier polls

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (row, k) of a TM x KC chunk in the no-swizzle K-major core-matrix layout:
// core matrix = 8 rows x 4 FP32 (16 B per row, 128 B); K-adjacent core matrices 128 B apart (LBO),
// 8-row groups 1024 B apart (SBO).
__device__ __forceinline__ uint32_t chunk_offset(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

// Shared-memory matrix descriptor (tcgen05): start address, LBO, SBO in 16-byte units, version 1 at bit 46,
// no swizzle (layout type 0 in bits 61-63).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo_bytes, uint32_t sbo_bytes) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo_bytes >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo_bytes >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor: D FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9, 10-12 = 2), both K-major,
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; returns false (and leaves the barrier as is) when the limit runs out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < WAIT_LIMIT; it++)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 consecutive accumulator columns of this thread's lane (row).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

// Operand rows: row q (0..127) of A starts at a_rows[q] (nullptr = zero row); K valid entries per row.
// Loads chunk c (K elements [c*KC, c*KC+KC)) of A and B into stage buffers with 128 threads.
__device__ __forceinline__ void load_chunk(uint32_t sA, uint32_t sB, const float* const* a_rows,
                                           const float* const* b_rows, int c, int K, const float* dummy) {
  // 128 rows x 8 16-byte pieces per operand = 1024 pieces; 8 per thread per operand
  for (int p = threadIdx.x; p < TM * (KC / 4); p += 128) {
    int row = p >> 3, piece = p & 7;
    int k = c * KC + piece * 4;
    int rem = K - k;
    int bytes = rem >= 4 ? 16 : (rem > 0 ? rem * 4 : 0);
    const float* ar = a_rows[row];
    const float* br = b_rows[row];
    uint32_t off = chunk_offset(row, piece * 4);
    cp_async16(sA + off, (ar && bytes) ? (const void*)(ar + k) : (const void*)dummy, ar ? bytes : 0);
    cp_async16(sB + off, (br && bytes) ? (const void*)(br + k) : (const void*)dummy, br ? bytes : 0);
  }
}

// Runs the whole K loop of one tile. smem: 4 * STAGE_BYTES (1024-aligned) then two mbarriers and the TMEM
// address slot. All 128 threads call it; afterwards the accumulator sits in TMEM at *tmem_out.
// Returns false if a bounded wait ran out (the caller reports GP_ERR_TIMEOUT and skips its epilogue).
__device__ __forceinline__ bool tile_mma(uint8_t* smem, const float* const* a_rows, const float* const* b_rows,
                                         int K, const float* dummy, uint32_t tmem_d) {
  const uint32_t base = smem_u32(smem);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 4 * STAGE_BYTES);
  const int nchunk = (K + KC - 1) / KC;
  const uint32_t idesc = idesc_tf32(TM, TN);
  uint32_t phase[2] = {0, 0};
  bool ok = true;
  load_chunk(base, base + 2 * STAGE_BYTES, a_rows, b_rows, 0, K, dummy);
  cp_async_commit();
  for (int c = 0; c < nchunk; c++) {
    const int s = c & 1;
    if (c + 1 < nchunk) {
      const int s1 = (c + 1) & 1;
      if (c >= 1) {   // chunk c-1 used stage s1: its instructions must have finished reading it
        if (!mbar_wait(&bars[s1], phase[s1])) ok = false;
        phase[s1] ^= 1;
      }
      load_chunk(base + s1 * STAGE_BYTES, base + (2 + s1) * STAGE_BYTES, a_rows, b_rows, c + 1, K, dummy);
      cp_async_commit();
      cp_async_wait_1();
    } else {
      cp_async_wait_all();
    }
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t sa = base + s * STAGE_BYTES, sb = base + (2 + s) * STAGE_BYTES;
#pragma unroll
      for (int kk = 0; kk < KC / 8; kk++) {
        uint64_t ad = smem_desc(sa + kk * 256, 128, 1024);
        uint64_t bd = smem_desc(sb + kk * 256, 128, 1024);
        mma_tf32(tmem_d, ad, bd, idesc, (c > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(&bars[s]);
    }
    __syncthreads();
  }
  // the last chunk's commit covers every earlier instruction of this thread
  const int sl = (nchunk - 1) & 1;
  if (!mbar_wait(&bars[sl], phase[sl])) ok = false;
  phase[sl] ^= 1;
  if (nchunk >= 2) {   // drain the other stage's last commit so both barriers end in a known phase
    const int so = sl ^ 1;
    if (!mbar_wait(&bars[so], phase[so])) ok = false;
  }
  tc_fence_after();
  return ok;
}

// ------------------------------------------------------------------------------------------------
// Split-TF32 variant: each FP32 operand x is split into hi = rn_tf32(x) and lo = rn_tf32(x - hi) while it is
// staged (global -> registers -> shared), and the tile accumulates A_lo B_hi^T + A_hi B_lo^T + A_hi B_hi^T
// (three K=8 instructions per step), which carries about 21 significant bits through the products instead of
// the 11 of one TF32 pass (the split of Ootomo and Yokota, 2022). One stage of four 16 KB buffers per chunk;
// several CTAs per SM overlap one another's loads and instructions.
constexpr int SPLIT_SMEM_BYTES = 4 * STAGE_BYTES + 1024;

__device__ __forceinline__ uint32_t to_tf32_bits(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return u;
}

__device__ __forceinline__ void split_store(uint8_t* hi, uint8_t* lo, uint32_t off, float4 v) {
  uint32_t h0 = to_tf32_bits(v.x), h1 = to_tf32_bits(v.y), h2 = to_tf32_bits(v.z), h3 = to_tf32_bits(v.w);
  uint32_t l0 = to_tf32_bits(v.x - __uint_as_float(h0)), l1 = to_tf32_bits(v.y - __uint_as_float(h1));
  uint32_t l2 = to_tf32_bits(v.z - __uint_as_float(h2)), l3 = to_tf32_bits(v.w - __uint_as_float(h3));
  *reinterpret_cast<uint4*>(hi + off) = make_uint4(h0, h1, h2, h3);
  *reinterpret_cast<uint4*>(lo + off) = make_uint4(l0, l1, l2, l3);
}

__device__ __forceinline__ float4 load4(const float* row, int k, int K) {
  if (!row || k >= K) return make_float4(0.f, 0.f, 0.f, 0.f);
  if (k + 4 <= K) return *reinterpret_cast<const float4*>(row + k);
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  v.x = row[k];
  if (k + 1 < K) v.y = row[k + 1];
  if (k + 2 < K) v.z = row[k + 2];
  return v;
}

// smem: A_hi, A_lo, B_hi, B_lo (STAGE_BYTES each, 1024-aligned base), then one mbarrier at +4*STAGE_BYTES.
__device__ __forceinline__ bool tile_mma_split3(uint8_t* smem, const float* const* a_rows, const float* const* b_rows,
                                                int K, uint32_t tmem_d) {
  uint8_t* aH = smem;
  uint8_t* aL = smem + STAGE_BYTES;
  uint8_t* bH = smem + 2 * STAGE_BYTES;
  uint8_t* bL = smem + 3 * STAGE_BYTES;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 4 * STAGE_BYTES);
  const uint32_t sAH = smem_u32(aH), sAL = smem_u32(aL), sBH = smem_u32(bH), sBL = smem_u32(bL);
  const int nchunk = (K + KC - 1) / KC;
  const uint32_t idesc = idesc_tf32(TM, TN);
  uint32_t phase = 0;
  bool ok = true;
  // registers of the chunk being staged: 8 16-byte pieces of A and of B per thread, all loads in flight
  // together; chunk c+1 is fetched while chunk c's instructions run
  constexpr int PER = TM * (KC / 4) / 128;
  float4 va[PER], vb[PER];
  auto fetch = [&](int c) {
#pragma unroll
    for (int it = 0; it < PER; it++) {
      int p = threadIdx.x + it * 128;
      int row = p >> 3, k = c * KC + (p & 7) * 4;
      va[it] = load4(a_rows[row], k, K);
      vb[it] = load4(b_rows[row], k, K);
    }
  };
  fetch(0);
  for (int c = 0; c < nchunk; c++) {
    if (c > 0) {   // the previous chunk's instructions must be done with the buffers
      if (!mbar_wait(bar, phase)) ok = false;
      phase ^= 1;
    }
#pragma unroll
    for (int it = 0; it < PER; it++) {
      int p = threadIdx.x + it * 128;
      uint32_t off = chunk_offset(p >> 3, (p & 7) * 4);
      split_store(aH, aL, off, va[it]);
      split_store(bH, bL, off, vb[it]);
    }
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < KC / 8; kk++) {
        const uint32_t o = kk * 256;
        uint64_t ah = smem_desc(sAH + o, 128, 1024), al = smem_desc(sAL + o, 128, 1024);
        uint64_t bh = smem_desc(sBH + o, 128, 1024), bl = smem_desc(sBL + o, 128, 1024);
        mma_tf32(tmem_d, al, bh, idesc, (c > 0 || kk > 0) ? 1u : 0u);
        mma_tf32(tmem_d, ah, bl, idesc, 1u);
        mma_tf32(tmem_d, ah, bh, idesc, 1u);
      }
      mma_commit(bar);
    }
    if (c + 1 < nchunk) fetch(c + 1);   // global loads overlap the tensor-core work of chunk c
    __syncthreads();
  }
  if (!mbar_wait(bar, phase)) ok = false;
  tc_fence_after();
  return ok;
}

}  // namespace tcg
