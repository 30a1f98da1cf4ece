// Inline-PTX helpers of the tcgen05 kernels (k_core_tc, k_level_tc): mbarriers,
// bulk copies, shared-memory matrix descriptors, MMA issue and commit, tensor
// memory loads and BF16 packing.
#pragma once

#include <cuda_bf16.h>

#include "tb_common.cuh"

namespace tb {
namespace tc {

constexpr long long SPIN_LIMIT = 1ll << 26;

TB_DEV uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

TB_DEV void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
TB_DEV void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
TB_DEV void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
TB_DEV bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
// Bounded wait: false if the phase did not complete within the limit, or (when
// `abort` is given) once another role of the block has given up.
TB_DEV bool mbar_wait(uint64_t *bar, uint32_t phase, const volatile int *abort = nullptr) {
    for (long long i = 0; i < SPIN_LIMIT; ++i) {
        if (mbar_try_wait(bar, phase)) return true;
        if (abort && (i & 255) == 255 && *abort) return false;
    }
    return false;
}
TB_DEV void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
TB_DEV void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
TB_DEV void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
TB_DEV void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 B apart (stride byte offset), descriptor version 1.
TB_DEV uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;               // leading byte offset (unused with a 128 B swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;     // stride byte offset
    d |= (uint64_t)1 << 46;               // version
    d |= (uint64_t)2 << 61;               // swizzle 128 B
    return d;
}
// Instruction descriptor, kind::f16: BF16 A and B (K-major), FP32 D, M = 128.
TB_HD uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
TB_DEV void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
TB_DEV void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// 32 consecutive accumulator columns of this warp's 32 TMEM lanes (one per thread)
TB_DEV void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// byte offset of (row, byte-in-row) in a 128 B-swizzled K-major tile
TB_HD uint32_t swz(uint32_t row, uint32_t byte) {
    return row * 128u + ((((byte >> 4) ^ (row & 7u)) << 4) | (byte & 15u));
}

TB_DEV uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}


// ---- 32-byte-swizzled K-major operands (one MMA K-step of 16 BF16 per row)
// An operand of `rows` rows and K = 16 s BF16 columns is stored as s K-step
// regions of rows x 32 B each.  Within a region the 16-byte halves of row r are
// swapped when bit 2 of r is set (the 32-byte swizzle on address bits 4 and 7),
// so a region must start on a 256-byte boundary.  With complex values stored as
// (re, im) BF16 pairs, a region row holds 8 complex columns.

// byte offset in a region of complex column c (0..7) of row r
TB_HD uint32_t sw32(uint32_t r, uint32_t c) {
    return r * 32u + ((((c >> 2) ^ (r >> 2)) & 1u) << 4) + ((c & 3u) << 2);
}
// Shared-memory matrix descriptor: K-major, 32-byte swizzle, 8-row groups 256 B
// apart (stride byte offset), descriptor version 1.
TB_DEV uint64_t sdesc32(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;               // leading byte offset (unused with a swizzle)
    d |= (uint64_t)(256 >> 4) << 32;      // stride byte offset
    d |= (uint64_t)1 << 46;               // version
    d |= (uint64_t)6 << 61;               // swizzle 32 B
    return d;
}
TB_DEV void sts32(uint32_t addr, uint32_t v) {
    asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
// (re, im) -> BF16 pairs hi = rn(v), lo = rn(v - hi), stored at hi_addr / lo_addr
TB_DEV void split_store(uint32_t hi_addr, uint32_t lo_addr, float re, float im) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(re - hf.x, im - hf.y);
    sts32(hi_addr, *reinterpret_cast<const uint32_t *>(&h));
    sts32(lo_addr, *reinterpret_cast<const uint32_t *>(&l));
}
// 16 consecutive accumulator columns of this warp's 32 TMEM lanes; complete
// after tmem_wait()
TB_DEV void tmem_ld16(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
TB_DEV void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// barrier of the 128 threads of warpgroup g (named barrier 1 + g)
TB_DEV void wg_sync(int g) { asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory"); }

// ---- interleaved split operands: each complex value as 8 bytes
// (hi re, hi im, lo re, lo im) in BF16, so a K-step region row (32 B, 16 BF16)
// holds 4 complex columns.  Byte offset in a region of complex column c (0..3)
// of row r, with the 32-byte swizzle:
TB_HD uint32_t sw32c(uint32_t r, uint32_t c) {
    return r * 32u + ((((c >> 1) ^ (r >> 2)) & 1u) << 4) + ((c & 1u) << 3);
}
// (re, im) -> {hi pair, lo pair}: hi = rn(v), lo = rn(v - hi)
TB_DEV uint2 split_pair(float re, float im) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(re - hf.x, im - hf.y);
    return make_uint2(*reinterpret_cast<const uint32_t *>(&h), *reinterpret_cast<const uint32_t *>(&l));
}

// ---- variants for kernels that order shared memory with explicit fences and
// barriers: no compiler memory clobber, so values held in registers (launch
// parameters, addresses) are not reloaded around every MMA or TMEM load
TB_DEV void mma_bf16_nc(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}
TB_DEV void tmem_ld16_nc(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
// tcgen05.wait::ld, then every register of r[0 .. 16 n) is tied to it, so no
// use of a loaded value is scheduled before the wait
template <int NCH>
TB_DEV void tmem_wait_regs(uint32_t *r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int i = 0; i < 16 * NCH; ++i) asm volatile("" : "+r"(r[i]));
}
}  // namespace tc
}  // namespace tb
