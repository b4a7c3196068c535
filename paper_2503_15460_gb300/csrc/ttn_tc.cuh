// Mode products of the complex64 bulk on the 5th-generation tensor cores
// (tcgen05, kind::tf32) with 3xTF32 split products and FP32 accumulation.
//
// A mode-k product out[l, p, r] = w sum_m M[p, m] in[l, m, r] is, for a
// tile of 128 fibres f = (l, r), the real GEMM
//     D[f, 2p + c'] = sum_{2m + c} A[f, 2m + c] B[2p + c', 2m + c]
// with A the fibres' interleaved (re, im) values and B the real 2 x 2 block
// form of w M:  B[2p, 2m] = Re, B[2p, 2m+1] = -Im, B[2p+1, 2m] = Im,
// B[2p+1, 2m+1] = Re of (w M)[p, m].  Each operand is split x = hi + lo
// with hi the TF32 rounding of x, and D = Ahi Bhi + Ahi Blo + Alo Bhi
// accumulates in FP32 in tensor memory (the Alo Blo term is below FP32
// rounding).  Operands are staged in shared memory in the K-major layout
// without swizzle (8-row x 16-byte core matrices); B stays resident for all
// tiles, A is staged in K-chunks.  One thread issues the MMAs, a tcgen05
// commit arrives on an mbarrier that every thread waits on (bounded), and
// warps 0-3 read the 128 x N accumulator rows back with tcgen05.ld.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kTcRows = 128;              // MMA M: fibres per tile
constexpr int kTcCols = 128;              // tensor-memory columns allocated (N <= 128)
constexpr long long kTcWaitLimit = 1ll << 22;   // try_wait rounds before an MMA is declared lost

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Shared-memory matrix descriptor: K-major, no swizzle.  lbo = byte distance
// between core matrices adjacent in K, sbo = between core matrices adjacent
// in the M (or N) dimension.
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;                // descriptor version of tcgen05
    return d;                              // base offset 0, no swizzle
}

// Instruction descriptor of kind::tf32: D in FP32, A and B TF32 and K-major.
__device__ __forceinline__ uint32_t tc_idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
        :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tc_mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool tc_mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_proxy_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// whole warp: allocate / free tensor-memory columns (address written to *dst)
__device__ __forceinline__ void tc_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(dst)), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols) : "memory");
}

// whole warp: 16 consecutive FP32 columns of this thread's accumulator row
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row, k) in a K-major no-swizzle tile with K
// extent kext (a multiple of 4): core matrix (row / 8, k / 4) at
// (row / 8) * sbo + (k / 4) * 128, sbo = (kext / 4) * 128.
__device__ __forceinline__ uint32_t tc_off(int row, int k, int kext) {
    return (uint32_t)((row >> 3) * (kext >> 2) * 128 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

struct TcShape {
    int n, Kp, Np, KC;                     // dimension, padded K and N, K chunk
    uint32_t b_bytes, a_bytes;             // one of hi / lo each
};

__device__ __forceinline__ TcShape tc_shape(int n, int stage_bytes) {
    TcShape s;
    s.n = n;
    s.Kp = ((2 * n + 7) / 8) * 8;
    s.Np = ((2 * n + 15) / 16) * 16;
    s.b_bytes = (uint32_t)s.Np * s.Kp * 4;
    int kc = (int)((stage_bytes - 2 * (int)s.b_bytes) / (2 * kTcRows * 4));
    kc = (kc / 8) * 8;
    s.KC = kc < s.Kp ? kc : s.Kp;
    s.a_bytes = (uint32_t)kTcRows * s.KC * 4;
    return s;
}

// Largest dimension the tensor-core product handles: N = 2n <= 128 columns.
__host__ __device__ constexpr int tc_max_dim() { return kTcCols / 2; }

// The resident B (hi and lo) plus an A chunk of at least one MMA K-step fit
// in stage_bytes.
__device__ __forceinline__ bool tc_fits(int n, int stage_bytes) {
    if (n < 1 || n > tc_max_dim()) return false;
    const int kp = ((2 * n + 7) / 8) * 8, np = ((2 * n + 15) / 16) * 16;
    return 2 * np * kp * 4 + 2 * kTcRows * 8 * 4 <= stage_bytes;
}

// Mode product by one thread block (NT threads, NT >= 128) over the fibre
// tiles tile0, tile0 + tstride, ...  smem: shared staging area of
// stage_bytes (128-byte aligned), taddr: kTcCols allocated tensor-memory
// columns, bar: an initialised mbarrier with its current phase.  Returns 0,
// or 1 when an MMA did not complete within the wait limit (nothing further
// is issued; the caller reports it).
template <int NT>
__device__ __noinline__ int tc_mode_prod(float2* out, const float2* in, int64_t L, int n, int64_t R, const float2* M, double2 w,
                            bool accumulate, unsigned char* smem, int stage_bytes, uint32_t taddr, uint64_t* bar,
                            uint32_t& phase, int64_t tile0, int64_t tstride) {
    const TcShape sh = tc_shape(n, stage_bytes);
    unsigned char* Bh = smem;
    unsigned char* Bl = Bh + sh.b_bytes;
    unsigned char* Ah = Bl + sh.b_bytes;
    unsigned char* Al = Ah + sh.a_bytes;
    // B = real block form of w M, split into TF32 hi / lo
    for (int i = threadIdx.x; i < sh.Np * sh.Kp; i += NT) {
        const int j = i / sh.Kp, k = i - j * sh.Kp;
        const int p = j >> 1, cp = j & 1, m = k >> 1, c = k & 1;
        float v = 0.f;
        if (p < n && m < n) {
            const float2 a = M[p * n + m];
            const double re = w.x * a.x - w.y * a.y, im = w.x * a.y + w.y * a.x;
            v = (float)(cp == 0 ? (c == 0 ? re : -im) : (c == 0 ? im : re));
        }
        const float h = tf32_rna(v);
        const uint32_t o = tc_off(j, k, sh.Kp);
        *(float*)(Bh + o) = h;
        *(float*)(Bl + o) = v - h;
    }
    const uint32_t idesc = tc_idesc_tf32(kTcRows, sh.Np);
    const int64_t F = L * R;
    const int64_t ntile = (F + kTcRows - 1) / kTcRows;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int err = 0;
    for (int64_t tile = tile0; tile < ntile && !err; tile += tstride) {
        const int64_t f0 = tile * kTcRows;
        for (int kc0 = 0; kc0 < sh.Kp && !err; kc0 += sh.KC) {
            const int kc = (sh.Kp - kc0) < sh.KC ? (sh.Kp - kc0) : sh.KC;
            // stage the A chunk: fibre f, interleaved column k in [kc0, kc0 + kc)
            for (int i = threadIdx.x; i < kTcRows * kc; i += NT) {
                int f, k;
                if (R == 1) { f = i / kc; k = i - f * kc; }            // fibre rows are contiguous
                else { k = i / kTcRows; f = i - k * kTcRows; }         // consecutive fibres are consecutive r
                const int kk = kc0 + k, m = kk >> 1, c = kk & 1;
                const int64_t g = f0 + f;
                float v = 0.f;
                if (g < F && m < n) {
                    const int64_t l = g / R, r = g - l * R;
                    const float2 x = in[(l * n + m) * R + r];
                    v = c == 0 ? x.x : x.y;
                }
                const float h = tf32_rna(v);
                const uint32_t o = tc_off(f, k, sh.KC);
                *(float*)(Ah + o) = h;
                *(float*)(Al + o) = v - h;
            }
            tc_fence_proxy_smem();
            __syncthreads();
            if (threadIdx.x == 0) {
                tc_fence_after();
                const uint32_t sa = (uint32_t)(sh.KC >> 2) * 128, sb = (uint32_t)(sh.Kp >> 2) * 128;
                for (int ks = 0; ks < kc; ks += 8) {
                    const uint32_t ao = (uint32_t)(ks >> 2) * 128, bo = (uint32_t)((kc0 + ks) >> 2) * 128;
                    const uint64_t ah = tc_smem_desc(smem_u32(Ah) + ao, 128, sa);
                    const uint64_t al = tc_smem_desc(smem_u32(Al) + ao, 128, sa);
                    const uint64_t bh = tc_smem_desc(smem_u32(Bh) + bo, 128, sb);
                    const uint64_t bl = tc_smem_desc(smem_u32(Bl) + bo, 128, sb);
                    const uint32_t first = (kc0 == 0 && ks == 0) ? 0u : 1u;
                    tc_mma_tf32(taddr, ah, bh, idesc, first);
                    tc_mma_tf32(taddr, ah, bl, idesc, 1u);
                    tc_mma_tf32(taddr, al, bh, idesc, 1u);
                }
                tc_commit(bar);
            }
            // every thread waits for the chunk's MMAs (bounded)
            long long it = 0;
            int late = 0;
            while (!tc_mbar_try_wait(bar, phase)) {
                if (++it > kTcWaitLimit) { late = 1; break; }
            }
            err = __syncthreads_or(late);        // one decision for the whole block
            phase ^= 1u;
            tc_fence_after();
        }
        if (err) break;
        // epilogue: warps 0-3 read rows 32 w .. 32 w + 31 of the accumulator
        if (warp < 4) {
            const int f = warp * 32 + lane;
            const int64_t g = f0 + f;
            const bool ok = g < F;
            int64_t l = 0, r = 0;
            if (ok) { l = g / R; r = g - l * R; }
            float2* dst = out + l * (int64_t)n * R + r;
            for (int c0 = 0; c0 < sh.Np; c0 += 16) {
                float v[16];
                tc_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
                if (!ok) continue;
#pragma unroll
                for (int q = 0; q < 16; q += 2) {
                    const int p = (c0 + q) >> 1;
                    if (p >= n) break;
                    float2 o = make_float2(v[q], v[q + 1]);
                    if (accumulate) { const float2 a = dst[(int64_t)p * R]; o.x += a.x; o.y += a.y; }
                    dst[(int64_t)p * R] = o;
                }
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    return err;
}

}  // namespace
