// nirc_tc.cuh -- tcgen05 / TMEM / mbarrier primitives (inline PTX, sm_100+).
//
// Operand layout used throughout: K-major, 128-byte swizzle.  A tile of R
// rows x 64 16-bit elements occupies R * 128 bytes; row r lives at
// (r / 8) * 1024 + (r % 8) * 128 and its 16-byte chunk c is stored at chunk
// position c ^ (r % 8).  Each 8-row group (1024 bytes) must start on a
// 1024-byte boundary.  A K = 16 step inside the 64-wide row is addressed by
// advancing the descriptor start by 32 bytes.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

namespace nirc {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (row, k) (k < 64, 16-bit elements) in a swizzled tile.
__host__ __device__ __forceinline__ uint32_t sw128_offset(uint32_t row, uint32_t k) {
    return (row >> 3) * 1024u + (row & 7u) * 128u + ((((k >> 3) ^ (row & 7u)) & 7u) << 4) + (k & 7u) * 2u;
}

// Byte offset of 8-bit element (row, k) (k < 64) in the same layout: a row
// keeps its 64 bytes in chunks 0-3 (16 elements each) of its 128-byte line.
__host__ __device__ __forceinline__ uint32_t sw128_offset_b8(uint32_t row, uint32_t k) {
    return (row >> 3) * 1024u + (row & 7u) * 128u + ((((k >> 4) ^ (row & 7u)) & 7u) << 4) + (k & 15u);
}

// Shared-memory matrix descriptor: K-major, SWIZZLE_128B, stride between
// 8-row groups 1024 bytes.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);  // start address
    d |= static_cast<uint64_t>(1u) << 16;                 // leading byte offset (unused for swizzled K-major)
    d |= static_cast<uint64_t>(1024u >> 4) << 32;         // stride byte offset
    d |= static_cast<uint64_t>(1u) << 46;                 // descriptor version
    d |= static_cast<uint64_t>(2u) << 61;                 // SWIZZLE_128B
    return d;
}

// Descriptor of an 8-row SWIZZLE_128B atom read as every 8-row group of an
// M = 128 operand (stride between 8-row groups 0): all 128 rows repeat it.
__device__ __forceinline__ uint64_t sdesc_rep8(uint32_t saddr) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
    d |= static_cast<uint64_t>(1u) << 16;
    d |= static_cast<uint64_t>(1u) << 46;
    d |= static_cast<uint64_t>(2u) << 61;
    return d;
}

// Shared-memory matrix descriptor without swizzling, K-major: 8-row x 16-byte
// core matrices stored as 128 contiguous bytes, the next core matrix along K
// `lbo` bytes further and the next 8-row group `sbo` bytes further.  The start
// may sit on any 16-byte core-matrix boundary (K offsets in steps of 8
// 16-bit elements).
__device__ __forceinline__ uint64_t sdesc_noswz(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
    d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
    d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
    d |= static_cast<uint64_t>(1u) << 46;  // descriptor version; swizzle mode 0 (none)
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulate, A/B type (0 = f16,
// 1 = bf16), both K-major, M x N.
__device__ __forceinline__ uint32_t idesc_f16(uint32_t ab_type, uint32_t M, uint32_t N) {
    return (1u << 4) | (ab_type << 7) | (ab_type << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// kind::f8f6f4 with both operands E4M3 (type code 0 in the instruction
// descriptor, so idesc_f16(0, M, N) describes it): K = 32 per instruction,
// i.e. 32 bytes of each K-major row, the same byte step as a kind::f16 K = 16.
__device__ __forceinline__ void mma_e4m3(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// The same MMA with A read from tensor memory: row m of A is TMEM lane m
// (relative to the lane base of the address), its K = 16 elements packed two
// per 32-bit column, the lower k in the low half (8 columns per MMA).
__device__ __forceinline__ void mma_f16_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t b, uint32_t idesc,
                                           uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n"
        :
        : "r"(tmem_d), "r"(tmem_a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void named_bar(uint32_t id, uint32_t threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for an mbarrier phase: gives up after ~2 s of device time or
// 2^28 polls and returns false (the caller records a timeout).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity) {
    if (mbar_try_wait(mbar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t it = 0; it < (1u << 28); ++it) {
        if (mbar_try_wait(mbar, parity)) return true;
        if ((it & 255u) == 255u && global_timer_ns() - t0 > 2000000000ull) break;
    }
    return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t holder_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(holder_smem), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 32 lanes x 64 columns of 32-bit accumulators (one row per thread).
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&v)[64]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, "
        "%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, "
        "%48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31]),
          "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]), "=r"(v[37]), "=r"(v[38]), "=r"(v[39]),
          "=r"(v[40]), "=r"(v[41]), "=r"(v[42]), "=r"(v[43]), "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]),
          "=r"(v[48]), "=r"(v[49]), "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]), "=r"(v[55]),
          "=r"(v[56]), "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]), "=r"(v[61]), "=r"(v[62]), "=r"(v[63])
        : "r"(taddr)
        : "memory");
}

// 32 lanes x 32 columns.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
}

// 32 lanes x 4 columns.
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&v)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                 : "r"(taddr)
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 32 lanes x 16 / 8 columns from registers (one row per thread).
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};"
        :
        : "r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
          "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                 :
                 : "r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, uint32_t v0, uint32_t v1, uint32_t v2, uint32_t v3) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};"
                 :
                 : "r"(taddr), "r"(v0), "r"(v1), "r"(v2), "r"(v3)
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// relu(lo), relu(hi) rounded to f16 (bf16) and packed, lo in the low half.
__device__ __forceinline__ uint32_t pack_relu_f16(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
__device__ __forceinline__ uint32_t pack_relu_bf16(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
// Four floats to E4M3 (round to nearest, saturating to +-448), element 0 in
// the lowest byte.
__device__ __forceinline__ uint32_t pack_e4m3x4(float x0, float x1, float x2, float x3) {
    uint16_t lo, hi;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(lo) : "f"(x1), "f"(x0));
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(hi) : "f"(x3), "f"(x2));
    return (uint32_t)lo | ((uint32_t)hi << 16);
}

__device__ __forceinline__ uint32_t pack_f16(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
__device__ __forceinline__ void sts16(uint32_t addr, uint16_t v) {
    asm volatile("st.shared.b16 [%0], %1;" ::"r"(addr), "h"(v) : "memory");
}
__device__ __forceinline__ uint4 lds128(uint32_t addr) {
    uint4 v;
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(addr)
                 : "memory");
    return v;
}
// Two packed 16-bit values (low half first) to FP32: bf16 by a shift, f16 by cvt.
template <uint32_t kBf16>
__device__ __forceinline__ float2 unpack2(uint32_t u) {
    if constexpr (kBf16) return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xFFFF0000u));
    return __half22float2(*reinterpret_cast<const __half2*>(&u));
}

}  // namespace tc

// Tensor-core weight image of the cache network (FP16/BF16/FP8 operands):
// 16-bit K-major swizzled matrices, the bias operands of the MMAs, then FP32
// biases and the FP8 weight scales.
namespace tcimg {
// Tensor-core weight image: 16-bit K-major swizzled matrices, then FP32 biases.
__host__ __device__ inline uint32_t off_w0pix() { return 0; }
__host__ __device__ inline uint32_t off_w0dir() { return 8192; }
__host__ __device__ inline uint32_t off_wh(uint32_t l) { return 16384 + 8192 * l; }
__host__ __device__ inline uint32_t off_wout(uint32_t hidden) { return 16384 + 8192 * (hidden - 1); }
// Biases as MMA operands: slot j (hidden layer j + 1, the output layer last)
// is K columns 16 (j % 4) .. + 15 of 64 x 64 tile j / 4; column 0 holds the
// 16-bit rounding b_hi of the bias, column 1 the remainder b_lo = b - b_hi,
// so that the MMA against an all-rows [1, 1, 0, ...] operand adds b to the
// accumulator with ~22 significant bits.  Then that 8-row ones atom.
__host__ __device__ inline uint32_t n_btiles(uint32_t hidden) { return (hidden + 3) / 4; }
__host__ __device__ inline uint32_t off_bmma(uint32_t hidden) { return off_wout(hidden) + 2048; }
__host__ __device__ inline uint32_t off_ones(uint32_t hidden) { return off_bmma(hidden) + 8192 * n_btiles(hidden); }
__host__ __device__ inline uint32_t off_bias(uint32_t hidden) { return off_ones(hidden) + 1024; }
__host__ __device__ inline uint32_t n_bias(uint32_t hidden) { return 64 + (hidden - 1) * 64 + 16; }
// FP8 weight scales s_w of the hidden layers (16 floats)
__host__ __device__ inline uint32_t off_scales(uint32_t hidden) { return off_bias(hidden) + n_bias(hidden) * 4; }
// End of the image the FP16 and FP8 kernels stage.
__host__ __device__ inline uint32_t bytes_hi(uint32_t hidden) { return off_scales(hidden) + 64; }
// Split BF16 operands: the remainders W - bf16(W) of the weight matrices,
// rounded to BF16, in a second region laid out like [0, off_wout + 2048).
__host__ __device__ inline uint32_t off_lo(uint32_t hidden) { return (bytes_hi(hidden) + 1023u) & ~1023u; }
__host__ __device__ inline uint32_t bytes_split(uint32_t hidden) { return off_lo(hidden) + off_wout(hidden) + 2048; }
}  // namespace tcimg

// 16-bit packing of A-tile rows (f16 or bf16).
template <uint32_t AB>
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    return AB ? tc::pack_bf16(lo, hi) : tc::pack_f16(lo, hi);
}
template <uint32_t AB>
__device__ __forceinline__ uint32_t pack2_relu(float lo, float hi) {
    return AB ? tc::pack_relu_bf16(lo, hi) : tc::pack_relu_f16(lo, hi);
}
template <uint32_t AB>
__device__ __forceinline__ uint16_t to16(float v) {
    return AB ? __bfloat16_as_ushort(__float2bfloat16_rn(v)) : __half_as_ushort(__float2half_rn(v));
}


// Swizzled 16-byte chunk c (8 elements) of row r of a tile.
__device__ __forceinline__ void sts_chunk(uint32_t tile, uint32_t r, uint32_t c, uint32_t d0, uint32_t d1, uint32_t d2,
                                          uint32_t d3) {
    tc::sts128(tile + (r >> 3) * 1024u + (r & 7u) * 128u + (((c ^ r) & 7u) << 4), d0, d1, d2, d3);
}

template <uint32_t AB>
__device__ __forceinline__ void sts_chunk8(uint32_t tile, uint32_t r, uint32_t c, const float* y) {
    sts_chunk(tile, r, c, pack2<AB>(y[0], y[1]), pack2<AB>(y[2], y[3]), pack2<AB>(y[4], y[5]), pack2<AB>(y[6], y[7]));
}

}  // namespace nirc
