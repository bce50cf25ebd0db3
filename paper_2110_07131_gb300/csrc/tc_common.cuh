// tcgen05 helpers shared by the batched filter (query.cu) and the index build
// (build_index.cu).  Device code only; include after rmips_internal.cuh.
#pragma once

#include "rmips_internal.cuh"

namespace rmips {

// ---------------------------------------------------------------------------
// tcgen05 (5th-generation tensor core) helpers: TMEM allocation, UMMA shared
// memory descriptors, MMA issue/commit and TMEM loads.
//
// Operand tiles use the K-major, non-swizzled canonical layout: the tile is cut
// into core matrices of 8 rows x 16 bytes (8 x 4 TF32 values); row r of a core
// matrix sits 16*r bytes from its start; core matrices adjacent along K are
// TC_LBO bytes apart and 8-row groups are TC_SBO bytes apart.
// ---------------------------------------------------------------------------
constexpr uint32_t TC_K = 64;                        // padded inner dimension (d <= 64)
// Relative error bound of a TF32 tensor-core inner product of float32 data,
// as a multiple of ||a|| ||b||: each operand is within 2^-10 of its float32
// value (10 fraction bits, any rounding), products of TF32 values are exact in
// float32, and the float32 accumulation over K = 64 terms (8 chained MMAs) is
// charged 65 * 2^-22 of sum |a_i b_i| <= ||a|| ||b||.
constexpr float TC_TF32_ERR = 0.00198f;              // >= 2^-9 + 2^-20 + 65 * 2^-22 * (1 + 2^-9)
constexpr uint32_t TC_LBO = 128;                     // next 16-byte K chunk
constexpr uint32_t TC_SBO = (TC_K / 4) * 128;        // next 8-row group (2048 bytes)

__host__ __device__ __forceinline__ uint32_t tc_off(uint32_t row, uint32_t k) {
  return (row >> 3) * TC_SBO + (k >> 2) * TC_LBO + (row & 7) * 16 + (k & 3) * 4;   // bytes
}

__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;                            // descriptor version of sm_100 family
  return d;                                          // base offset 0, no swizzle
}

// Instruction descriptor: D = F32, A = B = TF32, both K-major, shape M x N.
__host__ __device__ constexpr uint32_t tc_idesc_tf32(uint32_t M, uint32_t N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// kind::f16 (A = B = BF16 or FP16): 16-bit elements, a core matrix row holds
// 8 of them; the K = 64 tile is 8 chunks of 16 bytes, so 8-row groups are
// 1024 bytes apart, and one MMA consumes K = 16 (two chunks, 256 bytes).
constexpr uint32_t TC_SBO16 = (TC_K / 8) * 128;      // 1024 bytes

__host__ __device__ __forceinline__ uint32_t tc_off16(uint32_t row, uint32_t k) {
  return (row >> 3) * TC_SBO16 + (k >> 3) * TC_LBO + (row & 7) * 16 + (k & 7) * 2;   // bytes
}

// Instruction descriptor: D = F32, A = B = BF16 (bf16 = true) or FP16, K-major, M x N.
__host__ __device__ constexpr uint32_t tc_idesc_f16(uint32_t M, uint32_t N, bool bf16) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Operand layout of the batched tensor-core filter: rows of nstep K steps of
// 32 bytes (8 TF32 or 16 BF16 / FP16 values) in K-major core matrices
// (16-byte K chunks LBO = 128 bytes apart, 8-row groups SBO = 8 x 32 x nstep
// bytes apart); zeros between d and the row's K contribute nothing.  The
// index keeps its user tiles with rows of exactly the MMA's K (wf_nstep: for
// d = 50, 7 steps = K 56 for TF32, 4 = K 64 for the 16-bit kinds); in shared
// memory the filter uses rows of K = 64.
__host__ __device__ constexpr int wf_nstep(int tf32, int d) {
  return tf32 ? (d <= 32 ? 4 : (d <= 56 ? 7 : 8)) : (d <= 32 ? 2 : 4);
}
__host__ __device__ constexpr uint32_t wf_sbo(int nstep) { return 8u * 32u * (uint32_t)nstep; }
__host__ __device__ constexpr uint32_t wf_tile_bytes(int nstep) { return 128u * 32u * (uint32_t)nstep; }
// Byte offset of row r, K byte kb (a multiple of 16 for whole chunks).
__host__ __device__ __forceinline__ uint32_t wf_off(uint32_t r, uint32_t kb, uint32_t sbo) {
  return (r >> 3) * sbo + (kb >> 4) * TC_LBO + (r & 7) * 16 + (kb & 15);
}

// Operand kinds of the tensor-core filter: TF32 from float32 rows, or the
// index's BF16 / FP16 copy.
//
// tc_rel_err(kind) bounds |D - a.b| / (||a|| ||b||) for one MMA inner product
// D of two float32 vectors a, b over K <= 64, derived as follows.
//  1. Operand rounding: a_i' = a_i (1 + e_i), |e_i| <= u_in, where u_in is the
//     format's relative rounding error -- TF32 (10 fraction bits) 2^-10, which
//     covers truncation as well as rounding to nearest, BF16 (7 bits, rounded
//     to nearest) 2^-8, FP16 (10 bits, rounded to nearest) 2^-11.  So
//     |a_i' b_i' - a_i b_i| <= (2 u_in + u_in^2) |a_i b_i|.
//  2. Products: two TF32 / BF16 / FP16 significands have at most 22 bits, so
//     each a_i' b_i' is exact in float32.
//  3. Accumulation: a float32 sum of K terms that truncates at every step
//     errs by at most gamma = K 2^-23 / (1 - K 2^-23) times sum |a_i' b_i'|.
//     ASSUMPTION: the tensor core's accumulation of an MMA chain (internal
//     order, internal width, truncation) is within twice that of K + 1
//     sequential truncating float32 additions: 2 (K + 1) 2^-23 = 65 2^-22 for
//     K = 64.  Nothing documents the internal accumulation; the adversarial
//     tiles of the GPU tests check the whole bound, and it is the reason for
//     the factor 2.
//  4. sum |a_i' b_i'| <= (1 + u_in)^2 sum |a_i b_i| <= (1 + u_in)^2 ||a|| ||b||.
// Total: (2 u_in + u_in^2) + 65 2^-22 (1 + u_in)^2, rounded up:
//   TF32 2^-9 + 2^-20 + 65 2^-22 (1 + 2^-10)^2 = 0.0019696  -> 0.00198
//   BF16 2^-7 + 2^-16 + 65 2^-22 (1 + 2^-8)^2  = 0.0078436  -> 0.00788
//   FP16 2^-10 + 2^-22 + 65 2^-22 (1 + 2^-11)^2 = 0.0009923 -> 0.000995
// tc_abs_unit(kind) is the absolute rounding error of an operand below the
// format's normal range (FP16 subnormals: 2^-25; BF16 and TF32 share float32's
// range), which the filter charges separately.
enum : int { TCK_TF32 = 0, TCK_BF16 = 1, TCK_FP16 = 2 };
__host__ __device__ constexpr float tc_rel_err(int kind) {
  return kind == TCK_TF32 ? 0.00198f : (kind == TCK_BF16 ? 0.00788f : 0.000995f);
}
__host__ __device__ constexpr float tc_abs_unit(int kind) {
  return kind == TCK_FP16 ? 0x1p-25f : 0x1p-125f;
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 16 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
// 32 consecutive columns of this thread's TMEM lane and their largest value
// (tcgen05.ld with a max reduction; max is exact, so the fast Lemma 1 test
// keeps its rounding).
__device__ __forceinline__ float tmem_ld32_max(uint32_t taddr, float* v) {
  uint32_t r[32];
  float m;
  asm volatile(
      "tcgen05.ld.red.sync.aligned.32x32b.x32.max.f32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, %32, [%33];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
        "=f"(m)
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
  return m;
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }


}  // namespace rmips
