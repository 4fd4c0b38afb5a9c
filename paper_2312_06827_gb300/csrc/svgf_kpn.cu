// Learned part: a kernel-predicting network (KPN) that stands in for a-trous iterations 2-5.
//
//   features  10 channels from the pass-0 output and the G-buffer (BF16, padded to 16)
//   conv x4   3x3, 10 -> 32 -> 32 -> 32 -> 25 (ReLU between), BF16 operands, FP32 accumulation,
//             as implicit GEMMs on the 5th-generation tensor cores (tcgen05.mma, accumulators in
//             tensor memory); the same kernel computes the data gradient (dgrad) with the
//             flipped, transposed weights; the weight gradient (wgrad) is a second tensor-core
//             GEMM reduced over pixels (mma.sync m16n8k16 bf16, ldmatrix from padded tiles)
//   apply     softmax of the 25 logits = a 5x5 kernel per pixel (computed in the last layer's
//             epilogue, stored as 25 planes), applied to the pass-0 colour at dilation 1 and then
//             at dilation 4 (renormalised over in-image taps)
//   train     MSE in tone-mapped space against the plain pipeline's output, backward through
//             the applications, the softmax and the convolutions, Adam on FP32 master weights.
//
// Tensors: images [B][H][W][C] (pixel-major, channels contiguous); activations BF16 with 32
// channels (features 16); predicted kernels K and their gradients FP32 planar [25][B*H*W];
// colours float4.  Weights of the
// conv kernel: [9 taps][32 outputs][CI inputs] BF16 (inputs contiguous), tap = (dy+1)*3 + (dx+1).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>

#include "svgf_device.cuh"
#include "svgf_kpn.h"

namespace svgf {
namespace kpn {
namespace {

constexpr int TX = 16, TY = 8;        // conv output tile: 8 rows x 16 pixels, one row per warp

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4_t(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3,
                                          const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_addr(p)));
}

// D = A (16x16, row) * B (16x8, col) + D, BF16 operands, FP32 accumulators.
__device__ __forceinline__ void mma_bf16(float (&d)[4], unsigned a0, unsigned a1, unsigned a2,
                                         unsigned a3, unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
        "{%8, %9}, {%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float ex2_fast(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned*>(&v);
}
__device__ __forceinline__ unsigned pack_f16(float lo, float hi) {
    const __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const unsigned*>(&v);
}
__device__ __forceinline__ float2 unpack_f16(unsigned u) {
    return __half22float2(*reinterpret_cast<const __half2*>(&u));
}

// Copy a (TY+2) x (TX+2) halo tile of a [B][H][W][CI] BF16 image into shared memory (pixel
// stride CIP = CI + 8 to spread ldmatrix rows over the banks); zeros outside the image.
template <int CI, int CIP>
__device__ __forceinline__ void load_halo(__nv_bfloat16 (*s)[TX + 2][CIP], const __nv_bfloat16* in,
                                          int n, int H, int W, int x0, int y0, int tid, int nthr) {
    constexpr int CH = CI / 8;   // 16-byte chunks per pixel
    for (int i = tid; i < (TY + 2) * (TX + 2) * CH; i += nthr) {
        const int c = i % CH, px = i / CH;
        const int ly = px / (TX + 2), lx = px - ly * (TX + 2);
        const int gx = x0 + lx - 1, gy = y0 + ly - 1;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (gx >= 0 && gy >= 0 && gx < W && gy < H)
            v = *reinterpret_cast<const uint4*>(in + (((long)n * H + gy) * W + gx) * CI + c * 8);
        *reinterpret_cast<uint4*>(&s[ly][lx][c * 8]) = v;
    }
}

// ---- the 3x3 convolution on the 5th-generation tensor cores (tcgen05) ------------------------
// An output row segment = 128 consecutive pixels of one image row (M = 128) x 32 output channels.
// Input rows of pixels x0-1 .. x0+128 are staged in shared memory so that the K-major operand A
// of horizontal tap dx and channel chunk kc (K = 16) is a descriptor start address dx pixels
// further on -- no im2col copy.  32 channels: each pixel a 64-byte row in the 64-byte swizzled
// layout (8-row groups every 512 B), A starting at dx * 64 + kc * 32 bytes.  16 channels (the
// first layer): channel groups outermost, [group of 8 channels][pixel][8 channels], 8 x 16 B
// core matrices stacked along M every 128 B (SBO) and along K every 130 x 16 B (LBO).  Input row r enters output
// rows r+1, r and r-1 through the kernel rows dy = 0, 1, 2, so one MMA per (dx, kc) with the
// three kernel rows side by side along N (N = 96) adds row r's share to all three outputs: the
// weights sit as [dx][group][dy = 2, 1, 0][co][8] (B operand: SBO 128 B, LBO 96 x 16 B), and
// the output rows' FP32 accumulators are consecutive 32-column slots of a ring in tensor memory
// (a triple that wraps around the ring is issued as two MMAs).  One thread issues the MMAs of
// each input row and commits them to an mbarrier; an output row is complete once the row below
// it has been issued, and the four epilogue warps then read their 32 accumulator lanes (one
// pixel per thread, 32 channels) and zero the slot for its next use.
namespace tc {
constexpr int M = 128;
constexpr int HP = M + 2;
// Shared memory left free beyond the staged rows (none: the operand extents end inside them).
constexpr int kSlack = 0;
// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A and
// B (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits
// 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

// Shared-memory matrix descriptor, no swizzle: start address >> 4 (bits 0-13), leading-
// dimension byte offset >> 4 (bits 16-29, the K stride of core matrices), stride-dimension byte
// offset >> 4 (bits 32-45, the M/N stride of 8-row groups), descriptor version 1 (bit 46).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
__device__ __forceinline__ void mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t accumulate,
                                    uint32_t idesc = kIdesc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %3, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %4, p;\n\t}"
        ::"r"(dtmem), "l"(a), "l"(b), "r"(accumulate), "r"(idesc) : "memory");
}
// The instruction descriptor of kIdesc with N = n (a multiple of 16, at most 256) columns.
__device__ __forceinline__ uint32_t idesc_n(uint32_t n) {
    return (kIdesc & ~(0x3Fu << 17)) | ((n >> 3) << 17);
}
__device__ __forceinline__ void commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_addr(bar)) : "memory");
}
// The MMA (accumulating) and the commit issued by the lane elect.sync picks, for a whole warp
// walking the issue loop: its values are then warp-uniform, and the descriptors stay on the
// uniform datapath (one lane walking the loop inside a lane branch measured at about 240 cycles
// an MMA against 56 for N = 96).  In a converged warp elect.sync picks the same lane every
// time, so a commit tracks that lane's MMAs.
__device__ __forceinline__ void mma_elect(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc) {
    asm volatile(
        "{\n\t.reg .pred p, e;\n\tsetp.ne.u32 p, 1, 0;\n\telect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(dtmem), "l"(a), "l"(b), "r"(idesc) : "memory");
}
__device__ __forceinline__ void commit_elect(uint64_t* bar) {
    asm volatile(
        "{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}"
        ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_addr(slot)), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// Zeros into 32 lanes x 32 columns of tensor memory (the warp's lanes), complete on return.
__device__ __forceinline__ void st32_zero(uint32_t taddr) {
    const uint32_t z = 0;
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};"
                 ::"r"(taddr), "r"(z) : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
// 32 lanes x 32 columns of 32-bit accumulator: thread i of the warp gets lane (lane base + i).
__device__ __forceinline__ void ld32(uint32_t (&r)[32], uint32_t taddr) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count = 1) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// One arrival that also expects `bytes` of asynchronous copies to complete on the barrier.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// A TMA copy of one box of a 4-D tensor map (coordinates innermost first) into shared memory,
// completing its bytes on `bar`.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(smem_addr(dst)), "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}
// Named barrier ID (an immediate) over 128 threads (a group of four warps), returning whether
// `ok` held for all of them.
template <int ID>
__device__ __forceinline__ bool all_of_128(bool ok) {
    uint32_t r;
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.and.pred p, %2, 128, q;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(r) : "r"((uint32_t)ok), "n"(ID) : "memory");
    return r != 0;
}
// Bounded wait (about a second at most with the default number of tries) for the given phase of
// the barrier; false when it gave up.
constexpr int kWaitTries = 1 << 20;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int tries = kWaitTries) {
    for (int i = 0; i < tries; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, P;\n\t}"
            : "=r"(done) : "r"(smem_addr(bar)), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}
}  // namespace tc

// Bulk asynchronous shared -> global copy (16-byte aligned, size a multiple of 16), its group
// commit, and the waits for its source to be read / its writes to be done.
__device__ __forceinline__ void bulk_s2g(void* gdst, const void* ssrc, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                 ::"l"((unsigned long long)__cvta_generic_to_global(gdst)), "r"(smem_addr(ssrc)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// at most N of the bulk groups committed last still reading their source
template <int N = 0>
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// 16-byte asynchronous global -> shared copy; src_bytes = 0 fills the 16 bytes with zeros.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Staged input rows: a ring of kRing.
constexpr int kRing = 6;
// Accumulator slots (32 tensor-memory columns each) of the output-row ring.
constexpr unsigned kSlots = 8;
// Commit barriers of the input rows' MMAs.
constexpr unsigned kDone = 8;
// Output-row staging buffers of the epilogue (each M x 64 bytes): with two, an output row is
// written while the bulk store of the previous one still reads its buffer.  Two measured no
// faster at 1080p (nor a ring of 8 rows with 5 in flight), so one is kept.
constexpr int kOutBufs = 1;
// A staged 32-channel row in the 64-byte swizzled layout: 130 pixels x 64 bytes, padded to a
// multiple of the 512-byte swizzle pattern so that every ring slot starts on one.
constexpr int kRowSw64Bytes = 17 * 512;
// A 16-channel row in the 32-byte swizzled layout: 130 x 32 bytes padded to 17 x 256.
constexpr int kRowSw32Bytes = 17 * 256;
// Dynamic shared memory of a convolution block, at least: two blocks per SM, whose 2 x 8 slots
// fill the SM's 512 tensor-memory columns (a third block would wait in tcgen05.alloc).
constexpr size_t kMinConvSmem = 80 * 1024;

// One staged input row (image row gy of image n, pixels x0-1 .. x0+128, zeros outside the image,
// by a warp's 32 lanes with 16-byte cp.async) for CI = 32 in the 64-byte swizzled K-major
// layout: pixel px is a 64-byte row, its 16-byte chunk c (8 channels) stored at chunk
// c ^ ((px >> 1) & 3).  The tensor core applies the
// swizzle to the absolute shared-memory address bits (bits 4-5 ^= bits 7-8), so with the row
// slot 512-byte aligned, a tap shift of dx pixels is a start address dx * 64 bytes further on.
template <int NT>
__device__ __forceinline__ void tc_stage_row_sw64(unsigned char* dst, const __nv_bfloat16* __restrict__ in,
                                                  int n, int gy, int x0, int H, int W, int tid) {
    for (int i = tid; i < tc::HP * 4; i += NT) {
        const int kg = i % 4, px = i / 4, gx = x0 + px - 1;
        const bool ok = gx >= 0 && gx < W && gy >= 0 && gy < H;
        const __nv_bfloat16* src = ok ? in + (((long)n * H + gy) * W + gx) * 32 + kg * 8 : in;
        cp_async16(dst + px * 64 + ((kg ^ ((px >> 1) & 3)) << 4), src, ok ? 16u : 0u);
    }
    cp_async_commit();
}

// The same row for CI = 16 in the 32-byte swizzled K-major layout: pixel px is a 32-byte row,
// its chunk c stored at chunk c ^ ((px >> 2) & 1) (address bit 4 ^= bit 7), slots 256-byte
// aligned.
template <int NT>
__device__ __forceinline__ void tc_stage_row_sw32(unsigned char* dst, const __nv_bfloat16* __restrict__ in,
                                                  int n, int gy, int x0, int H, int W, int tid) {
    for (int i = tid; i < tc::HP * 2; i += NT) {
        const int kg = i & 1, px = i >> 1, gx = x0 + px - 1;
        const bool ok = gx >= 0 && gx < W && gy >= 0 && gy < H;
        const __nv_bfloat16* src = ok ? in + (((long)n * H + gy) * W + gx) * 16 + kg * 8 : in;
        cp_async16(dst + px * 32 + ((kg ^ ((px >> 2) & 1)) << 4), src, ok ? 16u : 0u);
    }
    cp_async_commit();
}

// Epilogue of one pixel: the 32 accumulated channels f (bias added) of pixel p.  EPI 1 writes
// the 25 kernel planes directly (a warp's 32 pixels are contiguous in each plane); EPI 0 / 2 write
// the pixel's 64 output bytes to `stage` (the tile's output row, stored in bulk afterwards).
template <int EPI>
__device__ __forceinline__ void tc_epilogue(float (&f)[32], long p, long npx,
                                            const __nv_bfloat16* __restrict__ mask, void* out,
                                            uint4* stage) {
    if (EPI == 1 || EPI == 3) {
        float mx = -INFINITY;
#pragma unroll
        for (int j = 0; j < 25; ++j) mx = fmaxf(mx, f[j]);
        float sum = 0.f;
#pragma unroll
        for (int j = 0; j < 25; ++j) {
            f[j] = ex2_fast((f[j] - mx) * 1.4426950408889634f);
            sum += f[j];
        }
        const float r = 1.0f / sum;
        if constexpr (EPI == 1) {
#pragma unroll
            for (int j = 0; j < 25; ++j) reinterpret_cast<float*>(out)[j * npx + p] = f[j] * r;
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) f[j] = j < 25 ? f[j] * r : 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                stage[q] = make_uint4(pack_f16(f[8 * q], f[8 * q + 1]), pack_f16(f[8 * q + 2], f[8 * q + 3]),
                                      pack_f16(f[8 * q + 4], f[8 * q + 5]), pack_f16(f[8 * q + 6], f[8 * q + 7]));
        }
        return;
    }
    if (EPI == 2) {
        const uint4* mk = reinterpret_cast<const uint4*>(mask + p * 32);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 m4 = mk[q];
            const unsigned mw[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const __nv_bfloat162 m2 = *reinterpret_cast<const __nv_bfloat162*>(&mw[h]);
                if (!(__low2float(m2) > 0.f)) f[8 * q + 2 * h] = 0.f;
                if (!(__high2float(m2) > 0.f)) f[8 * q + 2 * h + 1] = 0.f;
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) f[j] = fmaxf(f[j], 0.f);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        stage[q] = make_uint4(pack_bf16(f[8 * q], f[8 * q + 1]), pack_bf16(f[8 * q + 2], f[8 * q + 3]),
                              pack_bf16(f[8 * q + 4], f[8 * q + 5]), pack_bf16(f[8 * q + 6], f[8 * q + 7]));
}

// 3x3 convolution, 32 output channels: out[p][co] = epilogue(sum_{tap,ci} Wt[tap][co][ci] in[p+off][ci])
// EPI 0: + bias, ReLU, BF16 out.  EPI 1: + bias, then the softmax over the 25 logits of each
// pixel, written as 25 planes K[i][p] (FP32; npx = B*H*W).  EPI 2: x (mask[p][co] > 0), BF16 out
// (data gradient through the ReLU of the layer below).  EPI 3: the softmax of EPI 1 as FP16,
// pixel-major (25 weights and 7 zeros, 64 B per pixel, stored like a BF16 activation row; the
// inference form).  A block walks chunks of `chunk` output
// rows down one 128-pixel column of an image, reading input rows y0-1 .. y0+chunk.  Three roles,
// each walking the same chunks and rows (NG epilogue groups, 128 NG + 64 threads):
//   warp 4 NG + 1, the producer: copies each input row into a ring of kRing (one TMA copy a row,
//     completing on the slot's barrier) once the MMAs that read the slot's previous row have
//     completed;
//   warp 4 NG, the issuer (the whole warp walks the rows, one elected lane issues): per input
//     row, the MMAs into the output rows' accumulators;
//   warps 0 .. 4 NG - 1, the epilogue: group g takes the output rows of running index g modulo
//     NG; per output row, read its accumulator lanes, zero them, store.
// They meet at mbarriers, each waited for phase by phase (a parity wait must find its barrier at
// most one phase behind and not past the phase it waits for):
//   full[slot]     the producer's row has landed (TMA bytes)        -> the issuer;
//   rfree[slot]    the MMAs of the slot's row completed (commit)     -> the producer;
//   done[o % kDone] output row o complete: the MMAs of input row o + 1 (commit) -> the epilogue;
//   drained[acc]   the epilogue read and zeroed the accumulator slot -> the issuer.
// Rows take ring slots and output rows accumulator slots in the order the roles walk them (a
// running count), so a slot comes back kRing rows or kSlots output rows later.  The issuer can
// complete at most five output rows past the one the epilogue waits for (an accumulator slot
// is first written only after its previous output row was drained), below kDone = 8.
// Every wait is bounded: one that gives up sets kErrWaitGaveUp in *err and its side stops (the
// others' waits then run out too); the issuer commits once more to a barrier of its own and
// waits for it (all its MMAs done), and the block frees its tensor memory and returns.
template <int CI, int EPI, int NG>
__global__ void __launch_bounds__(128 * NG + 64, 2) k_conv3x3_tc(const __grid_constant__ CUtensorMap rows,
                                                       const __nv_bfloat16* __restrict__ in,
                                                       const __nv_bfloat16* __restrict__ wt,
                                                       const float* __restrict__ bias,
                                                       const __nv_bfloat16* __restrict__ mask,
                                                       void* out, int B, int H, int W, int chunk,
                                                       int* err) {
    using namespace tc;
    constexpr int KG = CI / 8;
    // rows and weights in the swizzled K-major layouts: CI = 32 rows of 64 bytes (slots of
    // 17 x 512 bytes), CI = 16 rows of 32 bytes (slots of 17 x 256 bytes)
    constexpr bool SW64 = CI == 32;     // else 32-byte swizzle
    constexpr bool SW64B = SW64;
    constexpr int RB = CI * 2;                       // bytes per pixel row (64 or 32)
    constexpr int ROW_BYTES = SW64 ? kRowSw64Bytes : kRowSw32Bytes;
    constexpr int W_BYTES = 9 * KG * 32 * 16, A_BYTES = kRing * ROW_BYTES, O_BYTES = NG * kOutBufs * M * 64;
    constexpr int NT = 128 * NG + 64;
    extern __shared__ __align__(1024) unsigned char tc_smem[];   // ring slots on 512-byte boundaries
    unsigned char* sw = tc_smem;
    unsigned char* sa = tc_smem + W_BYTES;
    uint4* so = reinterpret_cast<uint4*>(tc_smem + W_BYTES + A_BYTES);      // output rows [NG][kOutBufs][M][64 B]
    uint64_t* bar = reinterpret_cast<uint64_t*>(tc_smem + W_BYTES + A_BYTES + O_BYTES + kSlack);
    uint64_t* done = bar;                              // [kDone]
    uint64_t* full = done + kDone;                     // [kRing]
    uint64_t* rfree = full + kRing;                    // [kRing]
    uint64_t* drained = rfree + kRing;                 // [kSlots]
    uint64_t* fin = drained + kSlots;                  // the issuer's last commit
    uint32_t* tslot = reinterpret_cast<uint32_t*>(fin + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // weights [tap][co][ci] -> per dx the 96 rows (2 - dy) * 32 + co of the B operand, swizzled
    // like the input rows (64-byte rows for 32 channels, 32-byte rows for 16)
    for (int i = tid; i < 9 * 32 * KG; i += NT) {
        const int kg = i % KG, co = (i / KG) % 32, tap = i / (KG * 32), dy = tap / 3, dx = tap % 3;
        const int r = (2 - dy) * 32 + co;
        const int off = SW64B ? dx * 96 * 64 + r * 64 + ((kg ^ ((r >> 1) & 3)) << 4)
                              : dx * 96 * 32 + r * 32 + ((kg ^ ((r >> 2) & 1)) << 4);
        *reinterpret_cast<uint4*>(sw + off) = *reinterpret_cast<const uint4*>(wt + ((long)tap * 32 + co) * CI + kg * 8);
    }
    if (tid == 0) {
        for (unsigned i = 0; i < kDone; ++i) mbar_init(&done[i]);
        for (int r = 0; r < kRing; ++r) {
            mbar_init(&full[r], 1);
            mbar_init(&rfree[r]);
        }
        for (unsigned i = 0; i < kSlots; ++i) mbar_init(&drained[i], 128);
        mbar_init(fin);
    }
    if (warp == 0) tmem_alloc(tslot, 32 * kSlots);
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    if (warp < 4) {                    // every accumulator slot starts at zero
#pragma unroll 1
        for (unsigned sl = 0; sl < kSlots; ++sl) st32_zero(tmem + sl * 32u + ((uint32_t)(warp * 32) << 16));
    }
    fence_before();
    __syncthreads();
    fence_after();
    const long npx = (long)B * H * W;
    const int segs = (W + M - 1) / M, chunks_y = (H + chunk - 1) / chunk;
    const long total = (long)B * segs * chunks_y;

    if (warp == 4 * NG + 1) {
        // ---- the producer: each input row into the ring by one TMA copy (the tensor map's box
        // is the row's 130 pixels x CI channels, swizzled as the MMAs read it; pixels and rows
        // outside the image read as zeros) once the MMAs that read the slot's previous row have
        // completed; the copy completes on the slot's full barrier (one arrival, expected bytes)
        constexpr uint32_t kRowTx = (uint32_t)tc::HP * CI * 2;
        uint32_t used = 0, rpar = 0, ipar = 0;   // ipar: per slot, parity of the next copy's phase
        unsigned rs = 0;                // rows staged so far: the row's ring slot is rs % kRing
        bool fail = false;
        for (long c = blockIdx.x; c < total && !fail; c += gridDim.x) {
            const int n = (int)(c / ((long)segs * chunks_y));
            const int rc = (int)(c - (long)n * segs * chunks_y);
            const int seg = rc / chunks_y, y0 = (rc - seg * chunks_y) * chunk, x0 = seg * M;
            const int y1 = y0 + chunk < H ? y0 + chunk : H;
            for (int q = y0 - 1; q <= y1; ++q) {
                const int sl = (int)(rs++ % kRing);
                if ((used >> sl) & 1u) {        // the slot's previous row must have been read
                    const bool ok = __all_sync(0xffffffffu, mbar_wait(&rfree[sl], (rpar >> sl) & 1u));
                    rpar ^= 1u << sl;
                    if (!ok) {
                        fail = true;
                        break;
                    }
                }
                used |= 1u << sl;
                if (lane == 0) {
                    mbar_arrive_expect_tx(&full[sl], kRowTx);
                    tma_load_4d(sa + sl * ROW_BYTES, &rows, 0, x0 - 1, q, n, &full[sl]);
                }
                ipar ^= 1u << sl;
                __syncwarp();
            }
        }
        // the block's shared memory is released at its end: every copy issued must have landed
        for (int sl = 0; sl < kRing; ++sl)
            if ((used >> sl) & 1u) mbar_wait(&full[sl], ((ipar >> sl) & 1u) ^ 1u);
        if (fail && lane == 0) atomicOr(err, kErrWaitGaveUp);
    } else if (warp == 4 * NG) {
        // ---- the MMA issuer: the whole warp walks the rows, one elected lane issues
        {
            const uint32_t a0 = smem_addr(sa), b0 = smem_addr(sw);
            // descriptors of the ring's first slot and of the weights; an operand's descriptor
            // adds its byte offset / 16 to the start-address field (no carry: shared addresses
            // stay below 256 KB)
            // swizzled K-major operands: SBO = one 8-row group (512 or 256 bytes), swizzle mode at
            // bits 61-63 (64B = 4, 32B = 6); LBO is not used by these layouts
            const uint64_t A0 = SW64 ? (sdesc(a0, 16, 512) | (4ull << 61)) : (sdesc(a0, 16, 256) | (6ull << 61));
            const uint64_t B0 = SW64B ? (sdesc(b0, 16, 512) | (4ull << 61)) : (sdesc(b0, 16, 256) | (6ull << 61));
            unsigned nb = 0;           // input rows issued: ring slot nb % kRing
            unsigned obase = 0;        // output rows of earlier chunks (accumulator slot numbering)
            uint32_t fpar = 0;         // per ring slot: parity of the next row-ready phase
            uint32_t dused = 0, dpar = 0;   // per accumulator slot: used before, next drained parity
            bool fail = false;
            for (long c = blockIdx.x; c < total && !fail; c += gridDim.x) {
                const int rc = (int)(c % ((long)segs * chunks_y));
                const int y0 = (rc % chunks_y) * chunk;
                const int y1 = y0 + chunk < H ? y0 + chunk : H;
                for (int r = y0 - 1; r <= y1; ++r) {
                    const int sl = (int)(nb % kRing);
                    fail = !__all_sync(0xffffffffu, mbar_wait(&full[sl], (fpar >> sl) & 1u));
                    fpar ^= 1u << sl;
                    // output row r + 1 starts here: its slot's previous output must be drained
                    if (!fail && r + 1 <= y1 - 1) {
                        const unsigned ts = (obase + (unsigned)(r + 1 - y0)) % kSlots;
                        if ((dused >> ts) & 1u) {
                            fail = !__all_sync(0xffffffffu, mbar_wait(&drained[ts], (dpar >> ts) & 1u));
                            dpar ^= 1u << ts;
                        }
                        dused |= 1u << ts;
                    }
                    if (fail) break;
                    fence_after();
                    // output rows lo..hi of this chunk take input row r; output o uses kernel
                    // row dy = r - o + 1, stored as weight block 2 - dy = o - r + 1
                    const int lo = r - 1 > y0 ? r - 1 : y0, hi = r + 1 < y1 - 1 ? r + 1 : y1 - 1;
                    const int nblk = hi - lo + 1, blk0 = lo - r + 1;
                    const unsigned s0 = (obase + (unsigned)(lo - y0)) % kSlots;
                    const int first = nblk < (int)(kSlots - s0) ? nblk : (int)(kSlots - s0);
                    const uint32_t id1 = idesc_n(32u * first), id2 = idesc_n(32u * (nblk - first));
                    const uint64_t arow = A0 + (uint64_t)((sl * ROW_BYTES) >> 4);
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                        for (int kc = 0; kc < KG / 2; ++kc) {
                            const uint64_t a = arow + (uint64_t)((dx * RB + kc * 32) >> 4);
                            // B rows of block blk0 on: 32 rows per block (2048 B swizzled, 512 B plain)
                            const uint64_t bb = B0 + (uint64_t)((dx * 96 * RB + blk0 * 32 * RB + kc * 32) >> 4);
                            mma_elect(tmem + s0 * 32u, a, bb, id1);
                            if (first < nblk) mma_elect(tmem, a, bb + (uint64_t)((first * 32 * RB) >> 4), id2);
                        }
                    if (r - 1 >= y0) commit_elect(&done[(obase + (unsigned)(r - 1 - y0)) % kDone]);   // output r - 1 complete
                    commit_elect(&rfree[sl]);
                    ++nb;
                }
                obase += (unsigned)(y1 - y0);
            }
            if (fail && lane == 0) atomicOr(err, kErrWaitGaveUp);
            // the tensor memory is freed below: every MMA of the issuing lane must have completed
            if (nb > 0) {
                commit_elect(fin);
                mbar_wait(fin, 0u);
            }
        }
        __syncwarp();
    } else {
        // ---- warps 0 .. 4 NG - 1: the epilogue, NG groups of four warps, group g draining the
        // output rows whose running index is g modulo NG (with NG = 2 two rows drain at once;
        // kSlots and kDone are even, so each accumulator slot and done barrier has one group)
        const int g = warp >> 2, lx = (warp & 3) * 32 + lane;
        float bv[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) bv[j] = EPI == 2 ? 0.f : bias[j];
        unsigned obase = 0;             // output rows of earlier chunks
        unsigned nst = 0;               // rows this group has stored (its staging buffer)
        bool fail = false;
        for (long c = blockIdx.x; c < total && !fail; c += gridDim.x) {
            const int n = (int)(c / ((long)segs * chunks_y));
            const int rc = (int)(c - (long)n * segs * chunks_y);
            const int seg = rc / chunks_y, y0 = (rc - seg * chunks_y) * chunk, x0 = seg * M;
            const int y1 = y0 + chunk < H ? y0 + chunk : H;
            for (int o = y0; o < y1; ++o) {
                // output row o is complete with input row o + 1, whose MMAs commit to done[oi % kDone]
                const unsigned oi = obase + (unsigned)(o - y0);
                if ((int)(oi % NG) != g) continue;
                const bool ok = mbar_wait(&done[oi % kDone], (oi / kDone) & 1u);
                if (EPI != 1 && lx == 0) bulk_wait_read<kOutBufs - 1>();   // the row's buffer is free
                if (!(g == 0 ? all_of_128<2>(ok) : all_of_128<3>(ok))) {
                    if (lx == 0) atomicOr(err, kErrWaitGaveUp);
                    fail = true;
                    break;
                }
                fence_after();
                const unsigned ts = oi % kSlots;
                const uint32_t ta = tmem + ts * 32u + ((uint32_t)((warp & 3) * 32) << 16);
                uint32_t v[32];
                ld32(v, ta);
                st32_zero(ta);
                fence_before();
                mbar_arrive(&drained[ts]);
                const long prow = ((long)n * H + o) * W;
                const int x = x0 + lx;
                uint4* buf = so + (g * kOutBufs + nst % kOutBufs) * M * 4;
                if (x < W) {
                    float f[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) f[j] = __uint_as_float(v[j]) + bv[j];
                    tc_epilogue<EPI>(f, prow + x, npx, mask, out, buf + lx * 4);
                }
                if (EPI != 1) {
                    // the output pixels x0 .. min(x0 + 128, W) - 1 are contiguous: one bulk store
                    fence_proxy_async();
                    if (g == 0) asm volatile("bar.sync 4, 128;" ::: "memory");
                    else asm volatile("bar.sync 5, 128;" ::: "memory");
                    if (lx == 0) {
                        const int nv = W - x0 < M ? W - x0 : M;
                        bulk_s2g(reinterpret_cast<__nv_bfloat16*>(out) + (prow + x0) * 32, buf, (uint32_t)(nv * 64));
                    }
                }
                ++nst;
            }
            obase += (unsigned)(y1 - y0);
        }
        if (lx == 0) bulk_wait_all();
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) tmem_dealloc(tmem, 32 * kSlots);
}

// ---- the four layers in one kernel (inference) -------------------------------------------------
// The network's four convolutions in one pass, the activations never leaving the SM.  A block
// walks a chunk of output rows down one column segment; each layer's output row, once complete,
// goes from an epilogue (bias, ReLU, BF16) straight into the next layer's ring of input rows in
// shared memory, in the same 64-byte swizzled layout the per-layer kernel stages from global
// memory, and the last layer's softmax weights (FP16, pixel-major) are the only output.  Layer l
// has its own quarter of tensor memory: kNetSlots output-row accumulator slots of 32 columns.
// Columns: every layer computes the same 128 lanes, pixel x = s + lane.  Ring rows hold the
// pixels s - 1 .. s + 128 and the epilogues fill 1 .. 128 of them, so layer l is exact on lanes
// l .. 127 - l and a segment keeps lanes 3 .. 124 of the last layer: segments start kNetSeg = 122
// pixels apart (s = 122 seg - 3).  Outside the image the epilogue writes zeros, the zero padding
// each layer's input has in the per-layer form, so the result is that form's, bit for bit.
// Rows: for the chunk's output rows y0 .. y1 - 1, layer l reads rows y0 - 4 + l .. y1 + 3 - l
// (input k at y0 - 4 + l + k) and completes rows y0 - 3 + l .. y1 + 2 - l (output o at
// y0 - 3 + l + o, complete once input o + 2 is in); layer l's outputs are layer l + 1's inputs.
// Roles (20 warps): warp 16 + l issues layer l's MMAs (one elected lane), input row by input
// row, once the row is in its ring and the accumulator slot of the output row it starts was
// drained, and warp 16 also stages the feature rows into ring 0 (cp.async, kNetAhead rows ahead);
// epilogue warps 4l .. 4l + 3 drain layer l's output rows in order, each once its MMAs completed.
// One warp a layer issues and one group a layer drains, so the four layers' waits overlap: one
// thread issuing all four layers spent most of its time in its waits, and one group draining
// two layers set the pace at about 2,400 cycles a row each.  Barriers: per ring slot of layers
// 1-3 full (row written) and per ring slot rfree (its MMAs completed), per layer done (an output
// row's MMAs completed) and drained (an accumulator slot read), and a last commit per issuer;
// every wait is bounded as in the per-layer kernel.
constexpr int kNetSeg = 122;
constexpr int kNetRing0 = 4, kNetAhead = 2;       // feature rows (16 channels): ring, rows staged ahead
constexpr int kNetRing = 4;                       // input rows of layers 1-3
constexpr unsigned kNetSlots = 4;                 // 4 layers x 4 slots x 32 columns = 512
constexpr unsigned kNetDone = 4;
constexpr int kNetOutBufs = 2;
constexpr int kNetThreads = 20 * 32;
constexpr int kNetW0Bytes = 3 * 96 * 32, kNetW1Bytes = 3 * 96 * 64;
// shared memory: layers 1-3 weights, layer 0 weights, rings of layers 1-3, ring of layer 0,
// output staging, biases, barriers (every ring slot on a 512-byte boundary)
constexpr int kNetOffW0 = 3 * kNetW1Bytes;
constexpr int kNetOffRing = kNetOffW0 + kNetW0Bytes;
constexpr int kNetOffRing0 = kNetOffRing + 3 * kNetRing * kRowSw64Bytes;
constexpr int kNetOffOut = kNetOffRing0 + kNetRing0 * kRowSw32Bytes;
constexpr int kNetOffBias = kNetOffOut + kNetOutBufs * tc::M * 64;
constexpr int kNetOffBar = kNetOffBias + 4 * 32 * 4;
constexpr int kNetBars = kNetRing0 + 6 * kNetRing + 4 * (int)kNetDone + 4 * (int)kNetSlots + 4;
constexpr int kNetSmemBytes = kNetOffBar + kNetBars * 8 + 8;
static_assert(kNetOffRing % 512 == 0 && kNetOffRing0 % 512 == 0 && kNetOffOut % 16 == 0, "ring alignment");
static_assert(kNetRing >= 2 && kNetAhead < kNetRing0 && kNetAhead <= 2, "ring sizes");

struct NetWeights {
    const __nv_bfloat16* wt[4];
    const float* bias[4];
};

// Shared-memory state of the four-layer kernel.
struct NetSmem {
    unsigned char* ring0;      // [kNetRing0][kRowSw32Bytes]
    unsigned char* ring;       // [3][kNetRing][kRowSw64Bytes]: the input rows of layer l + 1
    unsigned char* sw0;        // layer 0 weights
    unsigned char* sw1;        // [3][kNetW1Bytes]
    uint4* so;                 // [kNetOutBufs][M][64 B]
    float* bias;               // [4][32]
    uint64_t *rfree0, *full, *rfree, *done, *drained, *fin;
};

// One chunk: image n, first kept row y0, rows output rows, first lane's pixel s.
struct NetChunk {
    int n, y0, rows, s;
};
__device__ __forceinline__ NetChunk net_chunk_of(long c, int H, int chunk, int segs, int chunks_y) {
    NetChunk ch;
    ch.n = (int)(c / ((long)segs * chunks_y));
    const int rc = (int)(c - (long)ch.n * segs * chunks_y);
    const int seg = rc / chunks_y;
    ch.y0 = (rc - seg * chunks_y) * chunk;
    ch.rows = (ch.y0 + chunk < H ? ch.y0 + chunk : H) - ch.y0;
    ch.s = seg * kNetSeg - 3;
    return ch;
}

// The MMAs of one input row of a layer (CI input channels): kernel-row blocks blk0.. of the
// weights into the accumulator slots s0.. of the layer's ring (two MMAs when the triple wraps).
template <int CI>
__device__ __forceinline__ void net_issue_row(uint32_t acc, uint64_t arow, uint64_t B0, int blk0, unsigned s0,
                                              int nblk) {
    using namespace tc;
    constexpr int RB = CI * 2;
    const int first = nblk < (int)(kNetSlots - s0) ? nblk : (int)(kNetSlots - s0);
    const uint32_t id1 = idesc_n(32u * first), id2 = idesc_n(32u * (nblk - first));
#pragma unroll
    for (int dx = 0; dx < 3; ++dx)
#pragma unroll
        for (int kc = 0; kc < CI / 16; ++kc) {
            const uint64_t a = arow + (uint64_t)((dx * RB + kc * 32) >> 4);
            const uint64_t bb = B0 + (uint64_t)((dx * 96 * RB + blk0 * 32 * RB + kc * 32) >> 4);
            mma_elect(acc + s0 * 32u, a, bb, id1);
            if (first < nblk) mma_elect(acc, a, bb + (uint64_t)((first * 32 * RB) >> 4), id2);
        }
}

// The issuer of layer L (a whole warp, one elected lane issuing): its input rows in order,
// across the block's chunks; layer 0's warp stages its rows too.
template <int L>
__device__ __forceinline__ void net_issuer(const NetSmem& sm, uint32_t tmem, const __nv_bfloat16* __restrict__ feats,
                                           int H, int W, int chunk, int segs, int chunks_y, long total, int* err) {
    using namespace tc;
    constexpr int CI = L == 0 ? 16 : 32;
    constexpr int NR = L == 0 ? kNetRing0 : kNetRing;
    constexpr int ROWB = L == 0 ? kRowSw32Bytes : kRowSw64Bytes;
    uint64_t* full = L == 0 ? nullptr : sm.full + (L - 1) * kNetRing;
    uint64_t* rfree = L == 0 ? sm.rfree0 : sm.rfree + (L - 1) * kNetRing;
    uint64_t* done = sm.done + L * kNetDone;
    uint64_t* drained = sm.drained + L * kNetSlots;
    // swizzled K-major operands: SBO = one 8-row group (256 or 512 bytes), swizzle mode at bits
    // 61-63 (32B = 6, 64B = 4)
    const uint64_t A0 = L == 0 ? (sdesc(smem_addr(sm.ring0), 16, 256) | (6ull << 61))
                               : (sdesc(smem_addr(sm.ring + (L - 1) * kNetRing * kRowSw64Bytes), 16, 512) | (4ull << 61));
    const uint64_t B0 = L == 0 ? (sdesc(smem_addr(sm.sw0), 16, 256) | (6ull << 61))
                               : (sdesc(smem_addr(sm.sw1 + (L - 1) * kNetW1Bytes), 16, 512) | (4ull << 61));
    const uint32_t acc = tmem + (uint32_t)(L * 32 * kNetSlots);
    unsigned nb = 0, ob = 0;
    uint32_t fpar = 0, dused = 0, dpar = 0;
    bool fail = false;
    // layer 0: this warp also stages the feature rows into ring 0, kNetAhead rows ahead of the
    // one it issues (rows y0 - 4 .. y1 + 3 of each chunk, in order across the block's chunks)
    long cs = blockIdx.x;
    int ks = 0;
    unsigned staged = 0;
    uint32_t used0 = 0, rpar0 = 0;
    const int lane = threadIdx.x & 31;
    auto stage_next = [&]() -> bool {
        if (cs >= total) return true;
        const NetChunk sc = net_chunk_of(cs, H, chunk, segs, chunks_y);
        const int sl = (int)(staged % kNetRing0);
        if ((used0 >> sl) & 1u) {           // the MMAs of the slot's previous row must be complete
            if (!__all_sync(0xffffffffu, mbar_wait(&sm.rfree0[sl], (rpar0 >> sl) & 1u))) return false;
            rpar0 ^= 1u << sl;
        }
        used0 |= 1u << sl;
        tc_stage_row_sw32<32>(sm.ring0 + sl * kRowSw32Bytes, feats, sc.n, sc.y0 - 4 + ks, sc.s, H, W, lane);
        ++staged;
        if (++ks == sc.rows + 8) {
            ks = 0;
            cs += gridDim.x;
        }
        return true;
    };
    for (long c = blockIdx.x; c < total && !fail; c += gridDim.x) {
        const NetChunk ch = net_chunk_of(c, H, chunk, segs, chunks_y);
        const int nin = ch.rows + 8 - 2 * L, nout = nin - 2;
        for (int k = 0; k < nin; ++k) {
            const int sl = (int)(nb % NR);
            if constexpr (L == 0) {
                while (!fail && staged < nb + 1 + kNetAhead && cs < total) fail = !stage_next();
                if (fail) break;
                // row nb's copies have landed once at most staged - nb - 1 later groups are pending
                const unsigned later = staged - nb - 1;
                if (later >= 2) cp_async_wait<2>();
                else if (later == 1) cp_async_wait<1>();
                else cp_async_wait<0>();
                fence_proxy_async();
                __syncwarp();
            } else {
                fail = !__all_sync(0xffffffffu, mbar_wait(&full[sl], (fpar >> sl) & 1u));
                fpar ^= 1u << sl;
            }
            // output row k starts here: its slot's previous row must be drained
            if (!fail && k < nout) {
                const unsigned ts = (ob + (unsigned)k) % kNetSlots;
                if ((dused >> ts) & 1u) {
                    fail = !__all_sync(0xffffffffu, mbar_wait(&drained[ts], (dpar >> ts) & 1u));
                    dpar ^= 1u << ts;
                }
                dused |= 1u << ts;
            }
            if (fail) break;
            fence_after();
            // outputs lo .. hi take input k; output o uses kernel row dy = k - o, stored as
            // weight block 2 - dy
            const int lo = k - 2 > 0 ? k - 2 : 0, hi = k < nout - 1 ? k : nout - 1;
            net_issue_row<CI>(acc, A0 + (uint64_t)((sl * ROWB) >> 4), B0, 2 - k + lo, (ob + (unsigned)lo) % kNetSlots,
                              hi - lo + 1);
            if (k >= 2) commit_elect(&done[(ob + (unsigned)(k - 2)) % kNetDone]);
            commit_elect(&rfree[sl]);
            ++nb;
        }
        ob += (unsigned)nout;
    }
    if (L == 0) cp_async_wait<0>();
    if (fail && (threadIdx.x & 31) == 0) atomicOr(err, kErrWaitGaveUp);
    // the tensor memory is freed at the end: every MMA of the issuing lane must have completed
    if (nb > 0) {
        commit_elect(&sm.fin[L]);
        mbar_wait(&sm.fin[L], 0u);
    }
}

// Named barrier over the 128 threads of epilogue group g (ids 2..5), returning whether `ok`
// held for all of them.
__device__ __forceinline__ bool net_all_of_group(bool ok, int g) {
    uint32_t r;
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.and.pred p, %2, 128, q;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(r) : "r"((uint32_t)ok), "r"(2 + g) : "memory");
    return r != 0;
}

// Epilogue state of one layer: output rows of earlier chunks, last-layer rows stored, and the
// use / parity bits of the next layer's ring slots.
struct NetEpi {
    unsigned ob, nst;
    uint32_t rused, rpar;
};

// Output row o of layer L in the chunk, by epilogue group g (thread lx = lane of tensor memory):
// once its MMAs completed, read and zero the accumulator slot, then bias and ReLU into the next
// layer's ring (zeros outside the image), or for the last layer the softmax, staged and stored
// in bulk (lanes 3 .. 124 of the segment).  False when a wait gave up.
template <int L>
__device__ __forceinline__ bool net_epi_item(const NetSmem& sm, NetEpi& e, const NetChunk& ch, int o, int g,
                                             uint32_t tmem, void* out, int H, int W, int lx, int* err) {
    using namespace tc;
    const unsigned oi = e.ob + (unsigned)o;
    bool ok = mbar_wait(&sm.done[L * kNetDone + oi % kNetDone], (oi / kNetDone) & 1u);
    const int q = (int)(oi % kNetRing);
    if (L < 3) {
        // the next layer's ring slot: the MMAs of its previous row must have completed
        if ((e.rused >> q) & 1u) {
            ok = mbar_wait(&sm.rfree[L * kNetRing + q], (e.rpar >> q) & 1u) && ok;
            e.rpar ^= 1u << q;
        }
        e.rused |= 1u << q;
    } else if (lx == 0) {
        bulk_wait_read<kNetOutBufs - 1>();   // the staging buffer is free
    }
    if (!net_all_of_group(ok, g)) {
        if (lx == 0) atomicOr(err, kErrWaitGaveUp);
        return false;
    }
    fence_after();
    const unsigned ts = oi % kNetSlots;
    const uint32_t ta = tmem + (uint32_t)(L * 32 * kNetSlots) + ts * 32u + ((uint32_t)((lx >> 5) * 32) << 16);
    uint32_t v[32];
    ld32(v, ta);
    st32_zero(ta);
    fence_before();
    mbar_arrive(&sm.drained[L * kNetSlots + ts]);
    const int x = ch.s + lx, y = ch.y0 - 3 + L + o;
    const float* bias = sm.bias + L * 32;
    float f[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) f[j] = __uint_as_float(v[j]) + bias[j];
    if constexpr (L < 3) {
        uint4 st[4] = {make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u),
                       make_uint4(0u, 0u, 0u, 0u)};
        if ((unsigned)x < (unsigned)W && (unsigned)y < (unsigned)H) tc_epilogue<0>(f, 0, 0, nullptr, nullptr, st);
        unsigned char* row = sm.ring + (L * kNetRing + q) * kRowSw64Bytes;
        const int px = lx + 1;
#pragma unroll
        for (int kg = 0; kg < 4; ++kg)
            *reinterpret_cast<uint4*>(row + px * 64 + ((kg ^ ((px >> 1) & 3)) << 4)) = st[kg];
        fence_proxy_async();
        mbar_arrive(&sm.full[L * kNetRing + q]);
    } else {
        uint4* buf = sm.so + (e.nst % kNetOutBufs) * tc::M * 4;
        tc_epilogue<3>(f, 0, 0, nullptr, nullptr, buf + lx * 4);
        fence_proxy_async();
        asm volatile("bar.sync 6, 128;" ::: "memory");
        if (lx == 0) {
            const int xs = ch.s + 3;
            const int nv = W - xs < kNetSeg ? W - xs : kNetSeg;
            if (nv > 0)
                bulk_s2g(reinterpret_cast<__half*>(out) + (((long)ch.n * H + y) * W + xs) * 32, buf + 3 * 4,
                         (uint32_t)(nv * 64));
        }
        ++e.nst;
    }
    return true;
}

__global__ void __launch_bounds__(kNetThreads, 1) k_kpn_net(const __nv_bfloat16* __restrict__ feats, NetWeights w,
                                                            void* out, int B, int H, int W, int chunk, int* err) {
    using namespace tc;
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    NetSmem sm;
    sm.sw1 = tc_smem;
    sm.sw0 = tc_smem + kNetOffW0;
    sm.ring = tc_smem + kNetOffRing;
    sm.ring0 = tc_smem + kNetOffRing0;
    sm.so = reinterpret_cast<uint4*>(tc_smem + kNetOffOut);
    sm.bias = reinterpret_cast<float*>(tc_smem + kNetOffBias);
    sm.rfree0 = reinterpret_cast<uint64_t*>(tc_smem + kNetOffBar);
    sm.full = sm.rfree0 + kNetRing0;
    sm.rfree = sm.full + 3 * kNetRing;
    sm.done = sm.rfree + 3 * kNetRing;
    sm.drained = sm.done + 4 * kNetDone;
    sm.fin = sm.drained + 4 * kNetSlots;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm.fin + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // weights [tap][co][ci] -> per dx the 96 rows (2 - dy) * 32 + co, swizzled like the rows
    for (int i = tid; i < 9 * 32 * 2; i += kNetThreads) {
        const int kg = i % 2, co = (i / 2) % 32, tap = i / 64, dy = tap / 3, dx = tap % 3;
        const int r = (2 - dy) * 32 + co;
        *reinterpret_cast<uint4*>(sm.sw0 + dx * 96 * 32 + r * 32 + ((kg ^ ((r >> 2) & 1)) << 4)) =
            *reinterpret_cast<const uint4*>(w.wt[0] + ((long)tap * 32 + co) * 16 + kg * 8);
    }
    for (int i = tid; i < 3 * 9 * 32 * 4; i += kNetThreads) {
        const int l = i / (9 * 32 * 4), j = i % (9 * 32 * 4);
        const int kg = j % 4, co = (j / 4) % 32, tap = j / 128, dy = tap / 3, dx = tap % 3;
        const int r = (2 - dy) * 32 + co;
        *reinterpret_cast<uint4*>(sm.sw1 + l * kNetW1Bytes + dx * 96 * 64 + r * 64 + ((kg ^ ((r >> 1) & 3)) << 4)) =
            *reinterpret_cast<const uint4*>(w.wt[l + 1] + ((long)tap * 32 + co) * 32 + kg * 8);
    }
    for (int i = tid; i < 128; i += kNetThreads) sm.bias[i] = w.bias[i >> 5][i & 31];
    // pixels 0 and 129 of the epilogue-filled rows are never written (they reach only the lanes
    // a segment does not keep): zeros
    for (int i = tid; i < 3 * kNetRing * 2 * 4; i += kNetThreads) {
        const int slot = i / 8, px = (i / 4) % 2 ? 129 : 0, kg = i % 4;
        *reinterpret_cast<uint4*>(sm.ring + slot * kRowSw64Bytes + px * 64 + (kg << 4)) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid == 0) {
        for (int r = 0; r < kNetRing0; ++r) mbar_init(&sm.rfree0[r]);
        for (int r = 0; r < 3 * kNetRing; ++r) {
            mbar_init(&sm.full[r], 128);
            mbar_init(&sm.rfree[r]);
        }
        for (unsigned i = 0; i < 4 * kNetDone; ++i) mbar_init(&sm.done[i]);
        for (unsigned i = 0; i < 4 * kNetSlots; ++i) mbar_init(&sm.drained[i], 128);
        for (int i = 0; i < 4; ++i) mbar_init(&sm.fin[i]);
    }
    if (warp == 0) tmem_alloc(tslot, 4 * 32 * kNetSlots);
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    if (warp < 4) {                    // every accumulator slot starts at zero
#pragma unroll 1
        for (unsigned sl = 0; sl < 4 * kNetSlots; ++sl) st32_zero(tmem + sl * 32u + ((uint32_t)(warp * 32) << 16));
    }
    fence_before();
    __syncthreads();
    fence_after();
    const int segs = (W + kNetSeg - 1) / kNetSeg, chunks_y = (H + chunk - 1) / chunk;
    const long total = (long)B * segs * chunks_y;

    if (warp >= 16) {
        // ---- the issuers, one warp a layer (one elected lane issues); warp 16 stages the features
        if (warp == 16) net_issuer<0>(sm, tmem, feats, H, W, chunk, segs, chunks_y, total, err);
        else if (warp == 17) net_issuer<1>(sm, tmem, feats, H, W, chunk, segs, chunks_y, total, err);
        else if (warp == 18) net_issuer<2>(sm, tmem, feats, H, W, chunk, segs, chunks_y, total, err);
        else net_issuer<3>(sm, tmem, feats, H, W, chunk, segs, chunks_y, total, err);
        __syncwarp();
    } else {
        // ---- the epilogues, warps 4l .. 4l + 3 for layer l, each output row in order
        const int g = warp >> 2, lx = (warp & 3) * 32 + lane;
        NetEpi e = {0, 0, 0, 0};
        bool ok = true;
        for (long c = blockIdx.x; c < total && ok; c += gridDim.x) {
            const NetChunk ch = net_chunk_of(c, H, chunk, segs, chunks_y);
            const int nout = ch.rows + 6 - 2 * g;
            for (int o = 0; o < nout && ok; ++o) {
                if (g == 0) ok = net_epi_item<0>(sm, e, ch, o, 0, tmem, out, H, W, lx, err);
                else if (g == 1) ok = net_epi_item<1>(sm, e, ch, o, 1, tmem, out, H, W, lx, err);
                else if (g == 2) ok = net_epi_item<2>(sm, e, ch, o, 2, tmem, out, H, W, lx, err);
                else ok = net_epi_item<3>(sm, e, ch, o, 3, tmem, out, H, W, lx, err);
            }
            e.ob += (unsigned)nout;
        }
        if (g == 3 && lx == 0) bulk_wait_all();
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) tmem_dealloc(tmem, 4 * 32 * kNetSlots);
}

// ---- two layers in one kernel ------------------------------------------------------------------
// The network as two kernels of two layers each (layers 0-1, then 2-3): the first layer's output
// rows go from their drain straight into the second layer's ring in shared memory, so of the three
// activations only the second layer's output crosses HBM.  With two layers a block, each layer
// has 8 accumulator slots (2 x 8 x 32 = the SM's 512 tensor-memory columns) as in the per-layer
// kernel, so an output row's slot comes back 8 rows later, and each layer's rows are drained by
// two groups of four warps, even rows and odd rows, so that two drains of a layer overlap.
// Columns: both layers compute the lanes x = s + lane; the second layer is exact on lanes 1 ..
// 126, and segments start kPairSeg = 126 pixels apart (s = 126 seg - 1).  Rows: for the chunk's
// output rows y0 .. y1 - 1, the first layer reads rows y0 - 2 .. y1 + 1 and completes y0 - 1 ..
// y1; the second reads those and completes y0 .. y1 - 1.  Roles (18 warps): warp 16 stages the
// input rows (cp.async, kPairAhead rows ahead) and issues the first layer's MMAs, warp 17 the
// second's (one elected lane each); drain warps 4g .. 4g + 3 take layer g >> 1, the rows whose
// running index has parity g & 1.  Zeros outside the image, accumulation order and epilogues as
// in the per-layer kernel, so the results are its results bit for bit.
constexpr int kPairSeg = 126;
constexpr int kPairRingIn = 4, kPairAhead = 2;
constexpr int kPairRing = 4;                      // even: all rows of a slot have the same parity
constexpr unsigned kPairSlots = 8;
constexpr unsigned kPairDone = 8;
constexpr int kPairOutBufs = 2;                   // output staging buffers a second-layer group
constexpr int kPairThreads = 18 * 32;
static_assert(kPairRing % 2 == 0 && kPairSlots % 2 == 0 && kPairDone % 2 == 0, "row parity owns slots");
static_assert(kPairAhead < kPairRingIn && kPairAhead <= 2, "ring sizes");

template <int LF>
struct PairCfg {
    static constexpr int CI0 = LF == 0 ? 16 : 32;                       // first layer's inputs
    static constexpr int ROW0 = LF == 0 ? kRowSw32Bytes : kRowSw64Bytes;
    static constexpr int W0B = 3 * 96 * CI0 * 2, W1B = 3 * 96 * 64;
    static constexpr int OFF_W0 = W1B;
    static constexpr int OFF_RIN = OFF_W0 + W0B;
    static constexpr int OFF_RMID = OFF_RIN + kPairRingIn * ROW0;
    static constexpr int OFF_OUT = OFF_RMID + kPairRing * kRowSw64Bytes;
    static constexpr int OFF_BIAS = OFF_OUT + 2 * kPairOutBufs * tc::M * 64;
    static constexpr int OFF_BAR = OFF_BIAS + 2 * 32 * 4;
    static constexpr int NBARS = kPairRingIn + 2 * kPairRing + 2 * (int)kPairDone + 2 * (int)kPairSlots + 2;
    static constexpr int SMEM_USED = OFF_BAR + NBARS * 8 + 8;
    // at least 120 KB, so that one block holds an SM (and its 512 tensor-memory columns)
    static constexpr int SMEM = SMEM_USED > 120 * 1024 ? SMEM_USED : 120 * 1024;
    static_assert(OFF_RIN % 512 == 0 && OFF_RMID % 512 == 0 && OFF_OUT % 16 == 0, "ring alignment");
};

struct PairSmem {
    unsigned char *rin, *rmid, *sw0, *sw1;
    uint4* so;                 // [2 groups][kPairOutBufs][M][64 B]
    float* bias;               // [2][32]
    uint64_t *rfree_in, *full, *rfree, *done, *drained, *fin;
};

__device__ __forceinline__ NetChunk pair_chunk_of(long c, int H, int chunk, int segs, int chunks_y) {
    NetChunk ch;
    ch.n = (int)(c / ((long)segs * chunks_y));
    const int rc = (int)(c - (long)ch.n * segs * chunks_y);
    const int seg = rc / chunks_y;
    ch.y0 = (rc - seg * chunks_y) * chunk;
    ch.rows = (ch.y0 + chunk < H ? ch.y0 + chunk : H) - ch.y0;
    ch.s = seg * kPairSeg - 1;
    return ch;
}

// The MMAs of one input row (CI input channels) into accumulator slots s0.. of a ring of
// kPairSlots (two MMAs when the triple wraps).
template <int CI>
__device__ __forceinline__ void pair_issue_row(uint32_t acc, uint64_t arow, uint64_t B0, int blk0, unsigned s0,
                                               int nblk) {
    using namespace tc;
    constexpr int RB = CI * 2;
    const int first = nblk < (int)(kPairSlots - s0) ? nblk : (int)(kPairSlots - s0);
    const uint32_t id1 = idesc_n(32u * first), id2 = idesc_n(32u * (nblk - first));
#pragma unroll
    for (int dx = 0; dx < 3; ++dx)
#pragma unroll
        for (int kc = 0; kc < CI / 16; ++kc) {
            const uint64_t a = arow + (uint64_t)((dx * RB + kc * 32) >> 4);
            const uint64_t bb = B0 + (uint64_t)((dx * 96 * RB + blk0 * 32 * RB + kc * 32) >> 4);
            mma_elect(acc + s0 * 32u, a, bb, id1);
            if (first < nblk) mma_elect(acc, a, bb + (uint64_t)((first * 32 * RB) >> 4), id2);
        }
}

// The issuer of layer J of the pair (a whole warp, one elected lane issuing); J = 0 also stages
// the input rows (rows y0 - 2 .. y1 + 1 of each chunk, kPairAhead rows ahead).
template <int LF, int J>
__device__ __forceinline__ void pair_issuer(const PairSmem& sm, uint32_t tmem, const __nv_bfloat16* __restrict__ in,
                                            int H, int W, int chunk, int segs, int chunks_y, long total, int* err) {
    using namespace tc;
    using C = PairCfg<LF>;
    constexpr int CI = J == 0 ? C::CI0 : 32;
    constexpr int NR = J == 0 ? kPairRingIn : kPairRing;
    constexpr int ROWB = J == 0 ? C::ROW0 : kRowSw64Bytes;
    constexpr uint64_t MODE = CI == 16 ? 6ull : 4ull;   // 32-byte / 64-byte swizzle
    constexpr uint32_t SBO = CI == 16 ? 256u : 512u;
    uint64_t* rfree = J == 0 ? sm.rfree_in : sm.rfree;
    uint64_t* done = sm.done + J * kPairDone;
    uint64_t* drained = sm.drained + J * kPairSlots;
    const uint64_t A0 = sdesc(smem_addr(J == 0 ? sm.rin : sm.rmid), 16, SBO) | (MODE << 61);
    const uint64_t B0 = sdesc(smem_addr(J == 0 ? sm.sw0 : sm.sw1), 16, SBO) | (MODE << 61);
    const uint32_t acc = tmem + (uint32_t)(J * 32 * kPairSlots);
    unsigned nb = 0, ob = 0;
    uint32_t fpar = 0, dused = 0, dpar = 0;
    bool fail = false;
    long cs = blockIdx.x;
    int ks = 0;
    unsigned staged = 0;
    uint32_t used0 = 0, rpar0 = 0;
    const int lane = threadIdx.x & 31;
    auto stage_next = [&]() -> bool {
        if (cs >= total) return true;
        const NetChunk sc = pair_chunk_of(cs, H, chunk, segs, chunks_y);
        const int sl = (int)(staged % kPairRingIn);
        if ((used0 >> sl) & 1u) {           // the MMAs of the slot's previous row must be complete
            if (!__all_sync(0xffffffffu, mbar_wait(&sm.rfree_in[sl], (rpar0 >> sl) & 1u))) return false;
            rpar0 ^= 1u << sl;
        }
        used0 |= 1u << sl;
        if constexpr (C::CI0 == 16) tc_stage_row_sw32<32>(sm.rin + sl * C::ROW0, in, sc.n, sc.y0 - 2 + ks, sc.s, H, W, lane);
        else tc_stage_row_sw64<32>(sm.rin + sl * C::ROW0, in, sc.n, sc.y0 - 2 + ks, sc.s, H, W, lane);
        ++staged;
        if (++ks == sc.rows + 4) {
            ks = 0;
            cs += gridDim.x;
        }
        return true;
    };
    for (long c = blockIdx.x; c < total && !fail; c += gridDim.x) {
        const NetChunk ch = pair_chunk_of(c, H, chunk, segs, chunks_y);
        const int nin = ch.rows + 4 - 2 * J, nout = nin - 2;
        for (int k = 0; k < nin; ++k) {
            const int sl = (int)(nb % NR);
            if constexpr (J == 0) {
                while (!fail && staged < nb + 1 + kPairAhead && cs < total) fail = !stage_next();
                if (fail) break;
                // row nb's copies have landed once at most staged - nb - 1 later groups are pending
                const unsigned later = staged - nb - 1;
                if (later >= 2) cp_async_wait<2>();
                else if (later == 1) cp_async_wait<1>();
                else cp_async_wait<0>();
                fence_proxy_async();
                __syncwarp();
            } else {
                fail = !__all_sync(0xffffffffu, mbar_wait(&sm.full[sl], (fpar >> sl) & 1u));
                fpar ^= 1u << sl;
            }
            // output row k starts here: its slot's previous row must be drained
            if (!fail && k < nout) {
                const unsigned ts = (ob + (unsigned)k) % kPairSlots;
                if ((dused >> ts) & 1u) {
                    fail = !__all_sync(0xffffffffu, mbar_wait(&drained[ts], (dpar >> ts) & 1u));
                    dpar ^= 1u << ts;
                }
                dused |= 1u << ts;
            }
            if (fail) break;
            fence_after();
            // outputs lo .. hi take input k; output o uses kernel row dy = k - o, stored as
            // weight block 2 - dy
            const int lo = k - 2 > 0 ? k - 2 : 0, hi = k < nout - 1 ? k : nout - 1;
            pair_issue_row<CI>(acc, A0 + (uint64_t)((sl * ROWB) >> 4), B0, 2 - k + lo, (ob + (unsigned)lo) % kPairSlots,
                               hi - lo + 1);
            if (k >= 2) commit_elect(&done[(ob + (unsigned)(k - 2)) % kPairDone]);
            commit_elect(&rfree[sl]);
            ++nb;
        }
        ob += (unsigned)nout;
    }
    if (J == 0) cp_async_wait<0>();
    if (fail && lane == 0) atomicOr(err, kErrWaitGaveUp);
    // the tensor memory is freed at the end: every MMA of the issuing lane must have completed
    if (nb > 0) {
        commit_elect(&sm.fin[J]);
        mbar_wait(&sm.fin[J], 0u);
    }
}

// Drain state of one group: output rows of earlier chunks, second-layer rows stored, and the use /
// parity bits of the second layer's ring slots it writes.
struct PairEpi {
    unsigned ob, nst;
    uint32_t rused, rpar;
};

// Output row o of pair layer J (running index oi, parity P) by drain group g: once its MMAs
// completed, read and zero the accumulator slot; the first layer's row goes (bias, ReLU, BF16,
// zeros outside the image) into the second layer's ring; the second layer's row is staged and
// stored in bulk (lanes 1 .. 126): bias, ReLU, BF16 for layer 1, the softmax as FP16 for layer
// 3.  False when a wait gave up.
template <int LF, int J>
__device__ __forceinline__ bool pair_epi_item(const PairSmem& sm, PairEpi& e, const NetChunk& ch, int o, int g,
                                              uint32_t tmem, void* out, int H, int W, int lx, int* err) {
    using namespace tc;
    const unsigned oi = e.ob + (unsigned)o;
    bool ok = mbar_wait(&sm.done[J * kPairDone + oi % kPairDone], (oi / kPairDone) & 1u);
    const int q = (int)(oi % kPairRing);
    if (J == 0) {
        if ((e.rused >> q) & 1u) {           // the MMAs of the slot's previous row must be complete
            ok = mbar_wait(&sm.rfree[q], (e.rpar >> q) & 1u) && ok;
            e.rpar ^= 1u << q;
        }
        e.rused |= 1u << q;
    } else if (lx == 0) {
        bulk_wait_read<kPairOutBufs - 1>();   // the staging buffer is free
    }
    if (!net_all_of_group(ok, g)) {
        if (lx == 0) atomicOr(err, kErrWaitGaveUp);
        return false;
    }
    fence_after();
    const unsigned ts = oi % kPairSlots;
    const uint32_t ta = tmem + (uint32_t)(J * 32 * kPairSlots) + ts * 32u + ((uint32_t)((lx >> 5) * 32) << 16);
    uint32_t v[32];
    ld32(v, ta);
    st32_zero(ta);
    fence_before();
    mbar_arrive(&sm.drained[J * kPairSlots + ts]);
    const int x = ch.s + lx, y = ch.y0 - 1 + J + o;
    const float* bias = sm.bias + J * 32;
    float f[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) f[j] = __uint_as_float(v[j]) + bias[j];
    if constexpr (J == 0) {
        uint4 st[4] = {make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u),
                       make_uint4(0u, 0u, 0u, 0u)};
        if ((unsigned)x < (unsigned)W && (unsigned)y < (unsigned)H) tc_epilogue<0>(f, 0, 0, nullptr, nullptr, st);
        unsigned char* row = sm.rmid + q * kRowSw64Bytes;
        const int px = lx + 1;
#pragma unroll
        for (int kg = 0; kg < 4; ++kg)
            *reinterpret_cast<uint4*>(row + px * 64 + ((kg ^ ((px >> 1) & 3)) << 4)) = st[kg];
        fence_proxy_async();
        mbar_arrive(&sm.full[q]);
    } else {
        const int p = g & 1;
        uint4* buf = sm.so + (p * kPairOutBufs + e.nst % kPairOutBufs) * tc::M * 4;
        if constexpr (LF == 0) tc_epilogue<0>(f, 0, 0, nullptr, nullptr, buf + lx * 4);
        else tc_epilogue<3>(f, 0, 0, nullptr, nullptr, buf + lx * 4);
        fence_proxy_async();
        if (p == 0) asm volatile("bar.sync 6, 128;" ::: "memory");
        else asm volatile("bar.sync 7, 128;" ::: "memory");
        if (lx == 0) {
            const int xs = ch.s + 1;
            const int nv = W - xs < kPairSeg ? W - xs : kPairSeg;
            if (nv > 0)
                bulk_s2g(reinterpret_cast<__nv_bfloat16*>(out) + (((long)ch.n * H + y) * W + xs) * 32, buf + 1 * 4,
                         (uint32_t)(nv * 64));
        }
        ++e.nst;
    }
    return true;
}

template <int LF>
__global__ void __launch_bounds__(kPairThreads, 1) k_kpn_pair(const __nv_bfloat16* __restrict__ in,
                                                              const __nv_bfloat16* __restrict__ w0,
                                                              const __nv_bfloat16* __restrict__ w1,
                                                              const float* __restrict__ b0, const float* __restrict__ b1,
                                                              void* out, int B, int H, int W, int chunk, int* err) {
    using namespace tc;
    using C = PairCfg<LF>;
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    PairSmem sm;
    sm.sw1 = tc_smem;
    sm.sw0 = tc_smem + C::OFF_W0;
    sm.rin = tc_smem + C::OFF_RIN;
    sm.rmid = tc_smem + C::OFF_RMID;
    sm.so = reinterpret_cast<uint4*>(tc_smem + C::OFF_OUT);
    sm.bias = reinterpret_cast<float*>(tc_smem + C::OFF_BIAS);
    sm.rfree_in = reinterpret_cast<uint64_t*>(tc_smem + C::OFF_BAR);
    sm.full = sm.rfree_in + kPairRingIn;
    sm.rfree = sm.full + kPairRing;
    sm.done = sm.rfree + kPairRing;
    sm.drained = sm.done + 2 * kPairDone;
    sm.fin = sm.drained + 2 * kPairSlots;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm.fin + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // weights [tap][co][ci] -> per dx the 96 rows (2 - dy) * 32 + co, swizzled like the rows
    constexpr int KG0 = C::CI0 / 8;
    for (int i = tid; i < 9 * 32 * KG0; i += kPairThreads) {
        const int kg = i % KG0, co = (i / KG0) % 32, tap = i / (KG0 * 32), dy = tap / 3, dx = tap % 3;
        const int r = (2 - dy) * 32 + co;
        const int off = C::CI0 == 32 ? dx * 96 * 64 + r * 64 + ((kg ^ ((r >> 1) & 3)) << 4)
                                     : dx * 96 * 32 + r * 32 + ((kg ^ ((r >> 2) & 1)) << 4);
        *reinterpret_cast<uint4*>(sm.sw0 + off) = *reinterpret_cast<const uint4*>(w0 + ((long)tap * 32 + co) * C::CI0 + kg * 8);
    }
    for (int i = tid; i < 9 * 32 * 4; i += kPairThreads) {
        const int kg = i % 4, co = (i / 4) % 32, tap = i / 128, dy = tap / 3, dx = tap % 3;
        const int r = (2 - dy) * 32 + co;
        *reinterpret_cast<uint4*>(sm.sw1 + dx * 96 * 64 + r * 64 + ((kg ^ ((r >> 1) & 3)) << 4)) =
            *reinterpret_cast<const uint4*>(w1 + ((long)tap * 32 + co) * 32 + kg * 8);
    }
    for (int i = tid; i < 64; i += kPairThreads) sm.bias[i] = i < 32 ? b0[i] : b1[i - 32];
    // pixels 0 and 129 of the second layer's ring rows are never written (they reach only lanes
    // 0 and 127, which a segment does not keep): zeros
    for (int i = tid; i < kPairRing * 2 * 4; i += kPairThreads) {
        const int slot = i / 8, px = (i / 4) % 2 ? 129 : 0, kg = i % 4;
        *reinterpret_cast<uint4*>(sm.rmid + slot * kRowSw64Bytes + px * 64 + (kg << 4)) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid == 0) {
        for (int r = 0; r < kPairRingIn; ++r) mbar_init(&sm.rfree_in[r]);
        for (int r = 0; r < kPairRing; ++r) {
            mbar_init(&sm.full[r], 128);
            mbar_init(&sm.rfree[r]);
        }
        for (unsigned i = 0; i < 2 * kPairDone; ++i) mbar_init(&sm.done[i]);
        for (unsigned i = 0; i < 2 * kPairSlots; ++i) mbar_init(&sm.drained[i], 128);
        for (int i = 0; i < 2; ++i) mbar_init(&sm.fin[i]);
    }
    if (warp == 0) tmem_alloc(tslot, 2 * 32 * kPairSlots);
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    if (warp < 4) {                    // every accumulator slot starts at zero
#pragma unroll 1
        for (unsigned sl = 0; sl < 2 * kPairSlots; ++sl) st32_zero(tmem + sl * 32u + ((uint32_t)(warp * 32) << 16));
    }
    fence_before();
    __syncthreads();
    fence_after();
    const int segs = (W + kPairSeg - 1) / kPairSeg, chunks_y = (H + chunk - 1) / chunk;
    const long total = (long)B * segs * chunks_y;
    if (warp >= 16) {
        if (warp == 16) pair_issuer<LF, 0>(sm, tmem, in, H, W, chunk, segs, chunks_y, total, err);
        else pair_issuer<LF, 1>(sm, tmem, in, H, W, chunk, segs, chunks_y, total, err);
        __syncwarp();
    } else {
        // drain groups: warps 4g .. 4g + 3 take layer g >> 1, rows of running parity g & 1
        const int g = warp >> 2, lx = (warp & 3) * 32 + lane, j = g >> 1, par = g & 1;
        PairEpi e = {0, 0, 0, 0};
        bool ok = true;
        for (long c = blockIdx.x; c < total && ok; c += gridDim.x) {
            const NetChunk ch = pair_chunk_of(c, H, chunk, segs, chunks_y);
            const int nout = ch.rows + 2 - 2 * j;
            for (int o = 0; o < nout && ok; ++o) {
                if (((e.ob + (unsigned)o) & 1u) != (unsigned)par) continue;
                if (j == 0) ok = pair_epi_item<LF, 0>(sm, e, ch, o, g, tmem, out, H, W, lx, err);
                else ok = pair_epi_item<LF, 1>(sm, e, ch, o, g, tmem, out, H, W, lx, err);
            }
            e.ob += (unsigned)nout;
        }
        if (j == 1 && lx == 0) bulk_wait_all();
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) tmem_dealloc(tmem, 2 * 32 * kPairSlots);
}

// Weight gradient of one layer: dW[co][tap][ci] += sum_p dZ[p][co] X[p + off(tap)][ci], over
// co < CO_REAL, ci < CI_REAL (the padded channels carry no parameters).  Nine warps, one tap each;
// every block walks tiles with a grid stride, keeps its partial sums in registers and adds them
// to dW once at the end.
template <int CI>
__global__ void __launch_bounds__(288) k_wgrad(const __nv_bfloat16* __restrict__ X,
                                               const __nv_bfloat16* __restrict__ dZ, float* dW,
                                               int B, int H, int W, int ci_real, int co_real) {
    constexpr int CIP = CI + 8, NT = CI / 8;
    __shared__ __align__(16) __nv_bfloat16 s_x[TY + 2][TX + 2][CIP];
    __shared__ __align__(16) __nv_bfloat16 s_dz[TY][TX][40];
    const int tid = threadIdx.x, lane = tid & 31, tap = tid >> 5;
    const int dy = tap / 3, dx = tap % 3;
    const int tiles_x = (W + TX - 1) / TX, tiles_y = (H + TY - 1) / TY;
    const int total = tiles_x * tiles_y * B;
    float acc[2][NT][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < NT; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
    const int mi = lane >> 3, ri = lane & 7;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int n = t / (tiles_x * tiles_y), r = t - n * tiles_x * tiles_y;
        const int y0 = (r / tiles_x) * TY, x0 = (r % tiles_x) * TX;
        __syncthreads();
        load_halo<CI, CIP>(s_x, X, n, H, W, x0, y0, tid, 288);
        for (int i = tid; i < TY * TX * 4; i += 288) {
            const int c = i & 3, px = i >> 2, ly = px / TX, lx = px % TX;
            const int gx = x0 + lx, gy = y0 + ly;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);   // pixels outside the image contribute nothing
            if (gx < W && gy < H)
                v = *reinterpret_cast<const uint4*>(dZ + (((long)n * H + gy) * W + gx) * 32 + c * 8);
            *reinterpret_cast<uint4*>(&s_dz[ly][lx][c * 8]) = v;
        }
        __syncthreads();
#pragma unroll 1
        for (int row = 0; row < TY; ++row) {            // k chunk: the 16 pixels of one row
            unsigned a[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)              // A = dZ^T: rows co, k pixels
                ldsm_x4_t(a[mt][0], a[mt][1], a[mt][2], a[mt][3],
                          &s_dz[row][ri + ((mi & 2) ? 8 : 0)][mt * 16 + ((mi & 1) ? 8 : 0)]);
#pragma unroll
            for (int np = 0; np < NT / 2; ++np) {       // B = shifted X: k pixels, n inputs
                unsigned b0, b1, b2, b3;
                ldsm_x4_t(b0, b1, b2, b3,
                          &s_x[row + dy][ri + ((mi & 1) ? 8 : 0) + dx][np * 16 + ((mi & 2) ? 8 : 0)]);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    mma_bf16(acc[mt][2 * np], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
                    mma_bf16(acc[mt][2 * np + 1], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b2, b3);
                }
            }
        }
    }
    const int g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int co = mt * 16 + g + ((e & 2) ? 8 : 0), ci = nt * 8 + 2 * tq + (e & 1);
                if (co < co_real && ci < ci_real)
                    atomicAdd(&dW[((long)co * 9 + tap) * ci_real + ci], acc[mt][nt][e]);
            }
}

// Bias gradient: db[co] += sum_p dZ[p][co] (co < co_real).
__global__ void k_bias_grad(const __nv_bfloat16* __restrict__ dZ, float* db, long npx, int co_real) {
    const int co = threadIdx.x & 31;
    float s = 0.f;
    for (long p = blockIdx.x * (long)(blockDim.x / 32) + (threadIdx.x >> 5); p < npx;
         p += (long)gridDim.x * (blockDim.x / 32))
        s += __bfloat162float(dZ[p * 32 + co]);
    __shared__ float red[8][32];
    red[threadIdx.x >> 5][co] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = 0.f;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) v += red[w][co];
        if (co < co_real) atomicAdd(&db[co], v);
    }
}

// ---------------------------------------------------------------- softmax + kernel application

// c_out(p) = sum_i K_i(p) c_in(p + d o_i) / sum_{i in image} K_i(p), K planar (K[i][p]).
// rgb_out: inverse tone map fused, written instead of c_out (channel 3 = var_src.w).
__global__ void k_apply(const float* __restrict__ K, const float4* __restrict__ c_in, float4* c_out,
                        int B, int H, int W, int d, Params P, float4* rgb_out,
                        const float4* __restrict__ var_src) {
    const long np = (long)B * H * W;
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    if (x >= W || y >= H) return;
    {
        const long base = (long)blockIdx.z * H * W;
        const long p = base + (long)y * W + x;
        float s = 0.f, r = 0.f, g = 0.f, b = 0.f;
#pragma unroll
        for (int ky = -2; ky <= 2; ++ky)
#pragma unroll
            for (int kx = -2; kx <= 2; ++kx) {
                const int qx = x + d * kx, qy = y + d * ky;
                if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
                const float k = __ldg(&K[((ky + 2) * 5 + (kx + 2)) * np + p]);
                const float4 c = __ldg(&c_in[base + (long)qy * W + qx]);
                s += k;
                r = fmaf(k, c.x, r);
                g = fmaf(k, c.y, g);
                b = fmaf(k, c.z, b);
            }
        const float inv = 1.0f / s;
        const float4 o = make_float4(r * inv, g * inv, b * inv, 0.f);
        if (rgb_out) {
            float3 c = make_float3(o.x, o.y, o.z);
            if (P.tonemap) {
                const float l = 0.2126f * c.x + 0.7152f * c.y + 0.0722f * c.z;
                float f;
                if (P.inverse_mode == 1) {
                    f = (1.0f + l) * P.inv_weight;
                } else {
                    float dd = 1.0f - P.luma_k * l;
                    dd = dd < 1e-6f ? 1e-6f : dd;
                    f = 1.0f / dd;
                }
                c = make_float3(c.x * f, c.y * f, c.z * f);
            }
            rgb_out[p] = make_float4(c.x, c.y, c.z, var_src ? var_src[p].w : 0.f);
        } else {
            c_out[p] = o;
        }
    }
}

// k_apply with the kernels as FP16, pixel-major (Kh[p][32], the first 25 used; conv EPI 3),
// the same sums in the same order.  A block of 32 x 8 threads takes 32 x 16 pixels (two a
// thread) and first copies their colour taps' window (the tile with a margin of 2 D) into shared
// memory, so that each of the 25 taps is read from there rather than through L1: at dilation 4
// the taps reach 8 pixels away and L1 serves few of them.
// The 25 FP16 kernel weights of pixel p (pixel-major, 64 bytes: 25 used) as floats.
__device__ __forceinline__ void load_kernel_h(const uint4* __restrict__ Kh, long p, float (&kv)[32]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint4 u = __ldg(&Kh[p * 4 + q]);
        const unsigned w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const float2 f = unpack_f16(w[h]);
            kv[8 * q + 2 * h] = f.x;
            kv[8 * q + 2 * h + 1] = f.y;
        }
    }
}

// One kernel application at pixel (x, y), dilation D: the K-weighted mean of the in-image taps
// (x + D kx, y + D ky), renormalised over them; the colours come from a shared-memory window
// `win` (pitch `pitch` float4) whose element (wx, wy) is the pixel (x, y).
template <int D>
__device__ __forceinline__ float3 apply_taps(const float (&kv)[32], const float4* win, int pitch, int wx, int wy,
                                             int x, int y, int W, int H) {
    float s = 0.f, r = 0.f, g = 0.f, b = 0.f;
#pragma unroll
    for (int ky = -2; ky <= 2; ++ky)
#pragma unroll
        for (int kx = -2; kx <= 2; ++kx) {
            const int qx = x + D * kx, qy = y + D * ky;
            if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
            const float k = kv[(ky + 2) * 5 + (kx + 2)];
            const float4 c = win[(wy + D * ky) * pitch + wx + D * kx];
            s += k;
            r = fmaf(k, c.x, r);
            g = fmaf(k, c.y, g);
            b = fmaf(k, c.z, b);
        }
    const float inv = 1.0f / s;
    return make_float3(r * inv, g * inv, b * inv);
}

// The inverse tone map of the library's Params (exact or the paper-literal form).
__device__ __forceinline__ float3 inverse_tm(const Params& P, float3 c) {
    if (P.tonemap) {
        const float l = 0.2126f * c.x + 0.7152f * c.y + 0.0722f * c.z;
        float f;
        if (P.inverse_mode == 1) {
            f = (1.0f + l) * P.inv_weight;
        } else {
            float dd = 1.0f - P.luma_k * l;
            dd = dd < 1e-6f ? 1e-6f : dd;
            f = 1.0f / dd;
        }
        c = make_float3(c.x * f, c.y * f, c.z * f);
    }
    return c;
}

template <int D>
__global__ void __launch_bounds__(256) k_apply_h(const uint4* __restrict__ Kh, const float4* __restrict__ c_in,
                                                 float4* c_out, int H, int W, Params P, float4* rgb_out,
                                                 const float4* __restrict__ var_src) {
    constexpr int TXp = 32, TYp = 16, HX = TXp + 4 * D, HY = TYp + 4 * D;
    __shared__ float4 tile[HY][HX];
    const int x0 = blockIdx.x * TXp, y0 = blockIdx.y * TYp;
    const long base = (long)blockIdx.z * H * W;
    for (int i = threadIdx.y * 32 + threadIdx.x; i < HX * HY; i += 256) {
        const int ly = i / HX, lx = i - ly * HX;
        const int gx = x0 - 2 * D + lx, gy = y0 - 2 * D + ly;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gx >= 0 && gx < W && gy >= 0 && gy < H) v = __ldg(&c_in[base + (long)gy * W + gx]);
        tile[ly][lx] = v;
    }
    __syncthreads();
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
        const int lx = threadIdx.x, ly = threadIdx.y + 8 * half;
        const int x = x0 + lx, y = y0 + ly;
        if (x >= W || y >= H) continue;
        const long p = base + (long)y * W + x;
        float kv[32];
        load_kernel_h(Kh, p, kv);
        const float3 o = apply_taps<D>(kv, &tile[0][0], HX, lx + 2 * D, ly + 2 * D, x, y, W, H);
        if (rgb_out) {
            const float3 c = inverse_tm(P, o);
            rgb_out[p] = make_float4(c.x, c.y, c.z, var_src ? var_src[p].w : 0.f);
        } else {
            c_out[p] = make_float4(o.x, o.y, o.z, 0.f);
        }
    }
}

// Backward of the second application and the loss: g2 = 2 (c2 - T) / (3 N); stores
// gK(p) = sum_c g2 (c1(q_i) - c2) / S2 and u(p) = g2 / S2; accumulates the squared error.
__global__ void k_bwd_apply2(const float* __restrict__ K, const float4* __restrict__ c1,
                             const float4* __restrict__ c2, const float4* __restrict__ T, float* gK,
                             float4* u, float* loss_sum, int B, int H, int W, float scale) {
    const long np = (long)B * H * W;
    float sq = 0.f;
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    if (x < W && y < H) {
        const long base = (long)blockIdx.z * H * W;
        const long p = base + (long)y * W + x;
        const float4 o = c2[p], t = T[p];
        const float e0 = o.x - t.x, e1 = o.y - t.y, e2 = o.z - t.z;
        sq += e0 * e0 + e1 * e1 + e2 * e2;
        const float g0 = scale * e0, g1 = scale * e1, g2 = scale * e2;
        float S = 0.f;
#pragma unroll
        for (int ky = -2; ky <= 2; ++ky)
#pragma unroll
            for (int kx = -2; kx <= 2; ++kx) {
                const int qx = x + 4 * kx, qy = y + 4 * ky;
                if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
                S += K[((ky + 2) * 5 + (kx + 2)) * np + p];
            }
        const float rS = 1.0f / S;
#pragma unroll
        for (int ky = -2; ky <= 2; ++ky)
#pragma unroll
            for (int kx = -2; kx <= 2; ++kx) {
                const int i = (ky + 2) * 5 + (kx + 2);
                const int qx = x + 4 * kx, qy = y + 4 * ky;
                float v = 0.f;
                if (qx >= 0 && qy >= 0 && qx < W && qy < H) {
                    const float4 q = c1[base + (long)qy * W + qx];
                    v = (g0 * (q.x - o.x) + g1 * (q.y - o.y) + g2 * (q.z - o.z)) * rS;
                }
                gK[i * np + p] = v;
            }
        u[p] = make_float4(g0 * rS, g1 * rS, g2 * rS, 0.f);
    }
    // block reduction of the squared error (blocks of 32 x 8 threads: one warp per row)
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    __shared__ float red[8];
    if (threadIdx.x == 0) red[threadIdx.y] = sq;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        float s = 0.f;
        for (int w = 0; w < 8; ++w) s += red[w];
        atomicAdd(loss_sum, s);
    }
}

// Gradient reaching c1: g1(q) = sum_i [p = q - 4 o_i in image] u(p) K_i(p); then the first
// application's kernel gradient gK(q) += sum_c g1 (c0(q + o_i) - c1(q)) / S1 and the softmax
// backward dz_j = K_j (gK_j - sum_i K_i gK_i), written as BF16 [p][32] (zeros past 25).
__global__ void k_bwd_apply1(const float* __restrict__ K, const float4* __restrict__ u,
                             const float4* __restrict__ c0, const float4* __restrict__ c1,
                             const float* __restrict__ gK, __nv_bfloat16* dz, int B, int H, int W) {
    const long np = (long)B * H * W;
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    if (x >= W || y >= H) return;
    {
        const long base = (long)blockIdx.z * H * W;
        const long q = base + (long)y * W + x;
        float g0 = 0.f, g1 = 0.f, g2 = 0.f;
#pragma unroll
        for (int ky = -2; ky <= 2; ++ky)
#pragma unroll
            for (int kx = -2; kx <= 2; ++kx) {
                const int px = x - 4 * kx, py = y - 4 * ky;
                if (px < 0 || py < 0 || px >= W || py >= H) continue;
                const long p = base + (long)py * W + px;
                const float k = K[((ky + 2) * 5 + (kx + 2)) * np + p];
                const float4 uu = u[p];
                g0 = fmaf(k, uu.x, g0);
                g1 = fmaf(k, uu.y, g1);
                g2 = fmaf(k, uu.z, g2);
            }
        const float4 o = c1[q];
        float S = 0.f;
        float Kq[25], gq[25];
#pragma unroll
        for (int i = 0; i < 25; ++i) {
            Kq[i] = K[i * np + q];
            gq[i] = gK[i * np + q];
        }
#pragma unroll
        for (int ky = -2; ky <= 2; ++ky)
#pragma unroll
            for (int kx = -2; kx <= 2; ++kx) {
                const int qx = x + kx, qy = y + ky;
                if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
                S += Kq[(ky + 2) * 5 + (kx + 2)];
            }
        const float rS = 1.0f / S;
#pragma unroll
        for (int ky = -2; ky <= 2; ++ky)
#pragma unroll
            for (int kx = -2; kx <= 2; ++kx) {
                const int qx = x + kx, qy = y + ky;
                if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
                const float4 c = c0[base + (long)qy * W + qx];
                gq[(ky + 2) * 5 + (kx + 2)] += (g0 * (c.x - o.x) + g1 * (c.y - o.y) + g2 * (c.z - o.z)) * rS;
            }
        float dot = 0.f;
#pragma unroll
        for (int i = 0; i < 25; ++i) dot = fmaf(Kq[i], gq[i], dot);
        unsigned* out = reinterpret_cast<unsigned*>(dz + q * 32);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int a = 2 * i, b = 2 * i + 1;
            const float va = a < 25 ? Kq[a] * (gq[a] - dot) : 0.f;
            const float vb = b < 25 ? Kq[b] * (gq[b] - dot) : 0.f;
            out[i] = pack_bf16(va, vb);
        }
    }
}

// ---------------------------------------------------------------- parameters

// From the flat FP32 parameters to the conv kernels' BF16 weights:
//  fwd[l]   [9][32][CIpad_l]: W_l[co][tap][ci] (zero for co >= 25 in layer 3, ci >= 10 in layer 0)
//  dgrad[l] [9][32][32]:      W_l[co][8 - tap][n = ci] transposed (l >= 1; zero for co >= 25)
//  bias[l]  [32]
__global__ void k_prep_weights(const float* __restrict__ prm, WeightPtrs w) {
    const int l = blockIdx.y;
    const int cin = cin_of(l), cout = cout_of(l), cip = cin_pad_of(l);
    const float* Wl = prm + param_offset(l);
    const float* bl = Wl + cout * 9 * cin;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 9 * 32 * cip; i += gridDim.x * blockDim.x) {
        const int ci = i % cip, co = (i / cip) % 32, tap = i / (cip * 32);
        const float v = (co < cout && ci < cin) ? Wl[((long)co * 9 + tap) * cin + ci] : 0.f;
        w.fwd[l][i] = __float2bfloat16_rn(v);
    }
    if (l >= 1)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 9 * 32 * 32; i += gridDim.x * blockDim.x) {
            const int co = i % 32, n = (i / 32) % 32, tap = i / (32 * 32);   // k = co, n = ci
            const float v = (co < cout && n < cin) ? Wl[((long)co * 9 + (8 - tap)) * cin + n] : 0.f;
            w.dgrad[l][i] = __float2bfloat16_rn(v);
        }
    if (blockIdx.x == 0 && threadIdx.x < 32) w.bias[l][threadIdx.x] = threadIdx.x < cout ? bl[threadIdx.x] : 0.f;
}

__global__ void k_adam(float* prm, const float* __restrict__ grad, float* m, float* v, int n,
                       float lr, float b1, float b2, float eps, float bc1, float bc2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float g = grad[i];
        const float mi = b1 * m[i] + (1.0f - b1) * g;
        const float vi = b2 * v[i] + (1.0f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        prm[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

// Features of the pass-0 output (tone-mapped colour, sqrt variance, log2 depth, octahedral
// normal, albedo), BF16 [H][W][16] (channels 10..15 zero).  cv in any storage precision.
template <class S>
__global__ void k_features_t(const typename S::Rec* __restrict__ cv, const float4* __restrict__ gbuf,
                             const float* __restrict__ albedo, __nv_bfloat16* feat, float4* c0,
                             int npx) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npx; p += gridDim.x * blockDim.x) {
        const float4 c = S::ld_cv(cv, p);
        const float4 g = gbuf[p];
        const float s = fabsf(g.x) + fabsf(g.y) + fabsf(g.z);
        float ox = g.x / s, oy = g.y / s;
        if (g.z < 0.f) {
            const float tx = (1.0f - fabsf(oy)) * (ox >= 0.f ? 1.f : -1.f);
            const float ty = (1.0f - fabsf(ox)) * (oy >= 0.f ? 1.f : -1.f);
            ox = tx;
            oy = ty;
        }
        float f[16] = {c.x, c.y, c.z, sqrtf(fmaxf(c.w, 0.f)), log2f(fmaxf(g.w, 1e-20f)), ox, oy,
                       albedo[3 * (long)p], albedo[3 * (long)p + 1], albedo[3 * (long)p + 2],
                       0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        uint4* o = reinterpret_cast<uint4*>(feat + (long)p * 16);
        o[0] = make_uint4(pack_bf16(f[0], f[1]), pack_bf16(f[2], f[3]), pack_bf16(f[4], f[5]), pack_bf16(f[6], f[7]));
        o[1] = make_uint4(pack_bf16(f[8], f[9]), 0u, 0u, 0u);
        if (c0) c0[p] = c;       // the pass-0 colour (and variance) the applications filter
    }
}

unsigned flat_grid(long n, int threads) {
    long b = (n + threads - 1) / threads;
    return (unsigned)(b > 152L * 32 ? 152L * 32 : (b < 1 ? 1 : b));
}

}  // namespace

cudaError_t prep_weights(const float* prm, const WeightPtrs& w, cudaStream_t s) {
    k_prep_weights<<<dim3(36, 4), 256, 0, s>>>(prm, w);
    return cudaGetLastError();
}

namespace {
// One thread initialises a single-arrival barrier and waits for its first phase, which no thread
// ever arrives at: the wait runs out after `tries` polls and the error bit is raised.
__global__ void k_wait_expiry(int tries, int* err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    tc::mbar_init(&bar);
    if (!tc::mbar_wait(&bar, 0u, tries)) atomicOr(err, kErrWaitGaveUp);
}
}  // namespace

cudaError_t wait_expiry_probe(int tries, int* err, cudaStream_t s) {
    if (tries < 1 || tries > tc::kWaitTries || err == nullptr) return cudaErrorInvalidValue;
    k_wait_expiry<<<1, 32, 0, s>>>(tries, err);
    return cudaGetLastError();
}

// Chunk length of a convolution launch: the B x segs columns of 128 pixels, each cut into
// chunks_y chunks, give at most one chunk to each of the grid's blocks (2 per SM), so that no
// block takes one more chunk than the others while they wait (with a fixed 16-row chunk a 1080p
// layer had 1020 chunks for 304 blocks: 108 blocks took four, the rest three); the chunk's two
// halo rows are then a small share of its rows.
static int conv_chunk(int B, int H, int W, int sm_count) {
    const long cols = (long)B * ((W + tc::M - 1) / tc::M);
    const long cap = (long)sm_count * 2;
    long per = cols >= cap ? 1 : cap / cols;            // chunks a column
    if (per > H) per = H;
    return (int)((H + per - 1) / per);
}

// The tensor map of a convolution's input [B][H][W][CI] BF16 for the producer's row copies: box
// CI channels x 130 pixels x 1 row x 1 image, in the swizzle the MMAs read (64-byte rows for 32
// channels, 32-byte rows for 16), zeros outside the tensor.  cuTensorMapEncodeTiled is reached
// through the runtime's driver entry point.
static cudaError_t encode_rows(CUtensorMap* map, const __nv_bfloat16* in, int CI, int B, int H, int W) {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !p) return cudaErrorNotSupported;
        fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    const cuuint64_t dims[4] = {(cuuint64_t)CI, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
    const cuuint64_t strides[3] = {(cuuint64_t)CI * 2, (cuuint64_t)W * CI * 2, (cuuint64_t)H * W * CI * 2};
    const cuuint32_t box[4] = {(cuuint32_t)CI, (cuuint32_t)tc::HP, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)in, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CI == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t conv(int layer, bool dgrad, const __nv_bfloat16* in, const WeightPtrs& w,
                 const __nv_bfloat16* mask, void* out, int B, int H, int W, int sm_count,
                 cudaStream_t s, int* err) {
    {
        const int chunk = conv_chunk(B, H, W, sm_count);
        const long tiles = (long)B * ((W + tc::M - 1) / tc::M) * ((H + chunk - 1) / chunk);
        const long cap = (long)sm_count * 2;
        const int grid = (int)(tiles < cap ? tiles : cap);
        // ng drain groups of four warps (two, except for the FP32-plane softmax, whose epilogue
        // needs more registers than 320 threads a block at two blocks a SM leave)
        auto launch = [&](auto kernel, int ci, int ng, const __nv_bfloat16* wt, const float* bias) {
            size_t smem = (size_t)9 * (ci / 8) * 32 * 16 + (size_t)kRing * (ci == 32 ? kRowSw64Bytes : kRowSw32Bytes) +
                          (size_t)ng * kOutBufs * tc::M * 64 + tc::kSlack + (kDone + 2 * kRing + kSlots + 1) * 8 + 8;
            if (smem < kMinConvSmem) smem = kMinConvSmem;
            cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            CUtensorMap rows;
            e = encode_rows(&rows, in, ci, B, H, W);
            if (e != cudaSuccess) return e;
            kernel<<<grid, 128 * ng + 64, smem, s>>>(rows, in, wt, bias, mask, out, B, H, W, chunk, err);
            return cudaGetLastError();
        };
        if (!dgrad) {
            if (layer == 0) return launch(k_conv3x3_tc<16, 0, 2>, 16, 2, w.fwd[0], w.bias[0]);
            if (layer < 3) return launch(k_conv3x3_tc<32, 0, 2>, 32, 2, w.fwd[layer], w.bias[layer]);
            if (layer == 3) return launch(k_conv3x3_tc<32, 1, 1>, 32, 1, w.fwd[3], w.bias[3]);
            return launch(k_conv3x3_tc<32, 3, 2>, 32, 2, w.fwd[3], w.bias[3]);   // layer 3, FP16 kernels
        }
        return launch(k_conv3x3_tc<32, 2, 2>, 32, 2, w.dgrad[layer], nullptr);
    }
}

// Chunk length of the four-layer kernel: one block a SM (its shared memory), the B x segs column
// segments cut into at most one chunk a block.
static int net_chunk(int B, int H, int W, int sm_count) {
    const long cols = (long)B * ((W + kNetSeg - 1) / kNetSeg);
    long per = cols >= sm_count ? 1 : sm_count / cols;
    if (per > H) per = H;
    return (int)((H + per - 1) / per);
}

cudaError_t net_forward(const __nv_bfloat16* feats, const WeightPtrs& w, void* Kh, int B, int H, int W,
                        int sm_count, cudaStream_t s, int* err) {
    if (B <= 0 || H <= 0 || W <= 0) return cudaSuccess;
    const int chunk = net_chunk(B, H, W, sm_count);
    const long tiles = (long)B * ((W + kNetSeg - 1) / kNetSeg) * ((H + chunk - 1) / chunk);
    const int grid = (int)(tiles < sm_count ? tiles : sm_count);
    cudaError_t e = cudaFuncSetAttribute(k_kpn_net, cudaFuncAttributeMaxDynamicSharedMemorySize, kNetSmemBytes);
    if (e != cudaSuccess) return e;
    NetWeights nw;
    for (int l = 0; l < 4; ++l) {
        nw.wt[l] = w.fwd[l];
        nw.bias[l] = w.bias[l];
    }
    k_kpn_net<<<grid, kNetThreads, kNetSmemBytes, s>>>(feats, nw, Kh, B, H, W, chunk, err);
    return cudaGetLastError();
}

// Chunk length of the two-layer kernels: one block a SM, at most one chunk a block.
static int pair_chunk(int B, int H, int W, int sm_count) {
    const long cols = (long)B * ((W + kPairSeg - 1) / kPairSeg);
    long per = cols >= sm_count ? 1 : sm_count / cols;
    if (per > H) per = H;
    return (int)((H + per - 1) / per);
}

cudaError_t net_pairs(const __nv_bfloat16* feats, const WeightPtrs& w, __nv_bfloat16* mid, void* Kh, int B, int H,
                      int W, int sm_count, cudaStream_t s, int* err) {
    if (B <= 0 || H <= 0 || W <= 0) return cudaSuccess;
    const int chunk = pair_chunk(B, H, W, sm_count);
    const long tiles = (long)B * ((W + kPairSeg - 1) / kPairSeg) * ((H + chunk - 1) / chunk);
    const int grid = (int)(tiles < sm_count ? tiles : sm_count);
    cudaError_t e = cudaFuncSetAttribute(k_kpn_pair<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, PairCfg<0>::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_kpn_pair<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, PairCfg<2>::SMEM);
    if (e != cudaSuccess) return e;
    k_kpn_pair<0><<<grid, kPairThreads, PairCfg<0>::SMEM, s>>>(feats, w.fwd[0], w.fwd[1], w.bias[0], w.bias[1], mid,
                                                               B, H, W, chunk, err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_kpn_pair<2><<<grid, kPairThreads, PairCfg<2>::SMEM, s>>>(mid, w.fwd[2], w.fwd[3], w.bias[2], w.bias[3], Kh,
                                                               B, H, W, chunk, err);
    return cudaGetLastError();
}

cudaError_t wgrad(int layer, const __nv_bfloat16* X, const __nv_bfloat16* dZ, float* grad_flat,
                  int B, int H, int W, int sm_count, cudaStream_t s) {
    const int tiles = ((W + TX - 1) / TX) * ((H + TY - 1) / TY) * B;
    const int grid = tiles < sm_count * 2 ? tiles : sm_count * 2;
    float* dW = grad_flat + param_offset(layer);
    float* db = dW + cout_of(layer) * 9 * cin_of(layer);
    if (layer == 0) k_wgrad<16><<<grid, 288, 0, s>>>(X, dZ, dW, B, H, W, cin_of(0), cout_of(0));
    else k_wgrad<32><<<grid, 288, 0, s>>>(X, dZ, dW, B, H, W, cin_of(layer), cout_of(layer));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long npx = (long)B * H * W;
    k_bias_grad<<<flat_grid(npx, 256), 256, 0, s>>>(dZ, db, npx, cout_of(layer));
    return cudaGetLastError();
}

cudaError_t apply(const float* K, const float4* c_in, float4* c_out, int B, int H, int W,
                  int dilation, const Params& P, float4* rgb_out, const float4* var_src, cudaStream_t s) {
    const dim3 grid((W + 31) / 32, (H + 7) / 8, B), block(32, 8);
    k_apply<<<grid, block, 0, s>>>(K, c_in, c_out, B, H, W, dilation, P, rgb_out, var_src);
    return cudaGetLastError();
}

cudaError_t apply_h(const void* Kh, const float4* c_in, float4* c_out, int B, int H, int W,
                    int dilation, const Params& P, float4* rgb_out, const float4* var_src, cudaStream_t s) {
    const dim3 grid((W + 31) / 32, (H + 15) / 16, B), block(32, 8);
    if (dilation == 1) k_apply_h<1><<<grid, block, 0, s>>>((const uint4*)Kh, c_in, c_out, H, W, P, rgb_out, var_src);
    else if (dilation == 4) k_apply_h<4><<<grid, block, 0, s>>>((const uint4*)Kh, c_in, c_out, H, W, P, rgb_out, var_src);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t backward_apply(const float* K, const float4* c0, const float4* c1, const float4* c2,
                           const float4* T, float* gK, float4* u, __nv_bfloat16* dz, float* loss_sum,
                           int B, int H, int W, cudaStream_t s) {
    const long np = (long)B * H * W;
    const float scale = 2.0f / (3.0f * (float)np);
    const dim3 grid((W + 31) / 32, (H + 7) / 8, B), block(32, 8);
    k_bwd_apply2<<<grid, block, 0, s>>>(K, c1, c2, T, gK, u, loss_sum, B, H, W, scale);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_bwd_apply1<<<grid, block, 0, s>>>(K, u, c0, c1, gK, dz, B, H, W);
    return cudaGetLastError();
}

cudaError_t adam(float* prm, const float* grad, float* m, float* v, float lr, float b1, float b2,
                 float eps, float bc1, float bc2, cudaStream_t s) {
    k_adam<<<flat_grid(kParamCount, 256), 256, 0, s>>>(prm, grad, m, v, kParamCount, lr, b1, b2, eps, bc1, bc2);
    return cudaGetLastError();
}

cudaError_t features(int prec, const void* cv, const float4* gbuf, const float* albedo,
                     __nv_bfloat16* feat, float4* c0, int npx, cudaStream_t s) {
    const unsigned g = flat_grid(npx, 256);
    switch (prec) {
        case 0: k_features_t<dev::StoreF32><<<g, 256, 0, s>>>((const float4*)cv, gbuf, albedo, feat, c0, npx); break;
        case 1: k_features_t<dev::Store16<false>><<<g, 256, 0, s>>>((const uint2*)cv, gbuf, albedo, feat, c0, npx); break;
        default: k_features_t<dev::Store16<true>><<<g, 256, 0, s>>>((const uint2*)cv, gbuf, albedo, feat, c0, npx); break;
    }
    return cudaGetLastError();
}

namespace {
// Per 32x32 tile: the population standard deviation of the pass-0 luminance (tone-mapped, the
// colour the network filters), two-pass; above the threshold -> flag = 1, counted.  Tiles with
// detail (edges, texture, contact shadows) are where the network's two narrow kernels depart
// from the wide, edge-stopped plain passes.
__global__ void __launch_bounds__(256) k_tile_flags(const float4* __restrict__ c0, int H, int W, float thr,
                                                    unsigned char* flags, int* count) {
    const int tx = blockIdx.x, ty = blockIdx.y;
    __shared__ float rs[256];
    __shared__ int rn[256];
    float l[4];
    bool in[4];
    float s = 0.f;
    int n = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = threadIdx.x + k * 256;
        const int x = tx * 32 + (i & 31), y = ty * 32 + (i >> 5);
        in[k] = x < W && y < H;
        l[k] = 0.f;
        if (in[k]) {
            const float4 c = c0[(long)y * W + x];
            l[k] = fmaf(0.0722f, c.z, fmaf(0.7152f, c.y, 0.2126f * c.x));
            s += l[k];
            ++n;
        }
    }
    rs[threadIdx.x] = s;
    rn[threadIdx.x] = n;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            rs[threadIdx.x] += rs[threadIdx.x + o];
            rn[threadIdx.x] += rn[threadIdx.x + o];
        }
        __syncthreads();
    }
    const float cnt = (float)rn[0];
    const float mean = rs[0] / cnt;
    __syncthreads();
    float ss = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float d = l[k] - mean;
        if (in[k]) ss = fmaf(d, d, ss);
    }
    rs[threadIdx.x] = ss;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) rs[threadIdx.x] += rs[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const unsigned char f = sqrtf(rs[0] / cnt) > thr ? 1 : 0;
        flags[ty * gridDim.x + tx] = f;
        if (f) atomicAdd(count, 1);
    }
}

// out = in dilated by r tiles (Chebyshev distance) over a tiles_x x tiles_y grid.
__global__ void k_dilate(const unsigned char* __restrict__ in, unsigned char* __restrict__ out,
                         int tiles_x, int tiles_y, int r) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= tiles_x * tiles_y) return;
    const int y = t / tiles_x, x = t - y * tiles_x;
    const int y0 = max(0, y - r), y1 = min(tiles_y - 1, y + r);
    const int x0 = max(0, x - r), x1 = min(tiles_x - 1, x + r);
    unsigned char v = 0;
    for (int yy = y0; yy <= y1 && !v; ++yy)
        for (int xx = x0; xx <= x1; ++xx) v |= in[yy * tiles_x + xx];
    out[t] = v;
}

// rgb_out <- plain for the pixels of flagged tiles.
__global__ void k_tile_select(const float4* __restrict__ plain, const unsigned char* __restrict__ flags,
                              float4* rgb_out, int H, int W) {
    const long n = (long)H * W;
    const int tiles_x = (W + 31) / 32;
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < n; p += (long)gridDim.x * blockDim.x) {
        const int x = (int)(p % W), y = (int)(p / W);
        if (flags[(y / 32) * tiles_x + x / 32]) rgb_out[p] = plain[p];
    }
}

__global__ void k_loss_finish(const float* sum, float* loss_out, float inv_n) {
    if (threadIdx.x == 0) *loss_out = *sum * inv_n;
}
}  // namespace

cudaError_t tile_flags(const float4* c0, int H, int W, float thr, unsigned char* flags, int* count,
                       cudaStream_t s) {
    k_tile_flags<<<dim3((W + 31) / 32, (H + 31) / 32), 256, 0, s>>>(c0, H, W, thr, flags, count);
    return cudaGetLastError();
}

cudaError_t tile_dilate(const unsigned char* in, unsigned char* out, int tiles_x, int tiles_y, int r,
                        cudaStream_t s) {
    const int n = tiles_x * tiles_y;
    k_dilate<<<(n + 255) / 256, 256, 0, s>>>(in, out, tiles_x, tiles_y, r);
    return cudaGetLastError();
}

cudaError_t tile_select(const float4* plain, const unsigned char* flags, float4* rgb_out, int H, int W,
                        cudaStream_t s) {
    k_tile_select<<<flat_grid((long)H * W, 256), 256, 0, s>>>(plain, flags, rgb_out, H, W);
    return cudaGetLastError();
}

cudaError_t loss_finish(const float* sum, float* loss_out, long n, cudaStream_t s) {
    k_loss_finish<<<1, 32, 0, s>>>(sum, loss_out, 1.0f / (3.0f * (float)n));
    return cudaGetLastError();
}

}  // namespace kpn
}  // namespace svgf
