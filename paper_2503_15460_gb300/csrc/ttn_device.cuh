// libttn device code: the sweep interpreter and its building blocks.
//
// Every routine below is written for a *team*: the threads that share one
// TTN instance.  Two team kinds exist:
//   Solo<NT>  one thread block of NT threads (many instances side by side,
//             one per block: the batched path for small and medium trees);
//   Clu       a thread-block cluster of up to 16 blocks of 512 threads (one
//             large instance spread over as many SMs: node tensors of the
//             paper's larger bond dimensions).
// Element loops run over the team's threads (tm.tid(), stride tm.nthr());
// tm.sync() separates dependent phases (__syncthreads() for Solo, a cluster
// barrier with release/acquire ordering for Clu).  Team-wide sums are
// reduced in a fixed order through distributed shared memory, so a cluster
// gives the same bits every run, and every block of a cluster takes the same
// control decisions (Krylov convergence, substeps, ranks) from identical
// values.
//
// T is the bulk element type: double2 (complex128 mode) or float2 (mixed
// mode).  Scalars that steer the algorithm -- Krylov coefficients, norms,
// the small projected exponential, Householder scalars -- are FP64 in both
// modes, and the QR works on an FP64 copy of the matricised tensor.
//
// This header is included by one translation unit per kernel variant; its
// contents have internal linkage.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ttn_program.h"
#include "ttn_tc.cuh"

// Builds with the tcgen05 mode product in the sweep kernel define this to 1.
#ifndef TTN_WITH_TC
#define TTN_WITH_TC 0
#endif

namespace {

namespace cg = cooperative_groups;

constexpr int kMaxWarps = 16;
// Dynamic shared memory: a staging area for operator matrices and tiles.
// Cluster blocks have a second area of the same size for cross-block
// partial sums.
constexpr int kStageBytes = 64 * 1024;
constexpr int kStageBytesClu = 2 * kStageBytes;
extern __shared__ __align__(16) unsigned char dyn_smem[];

// Algorithmic floating-point operations of the instance (complex multiply-add
// = 8), accumulated by thread 0 of the team's first block and flushed to the
// instance counter at exit.
__shared__ double s_flops;
// The part of them executed in FP64 arithmetic (element type complex128).
__shared__ double s_flops64;
// 1 in the block that counts (rank 0 of its team).
__shared__ int s_count;
template <class T>
__device__ __forceinline__ void count_flops_t(double f) {
    if (threadIdx.x == 0 && s_count) {
        s_flops += f;
        if (sizeof(T) == 16) s_flops64 += f;
    }
}

// Mode-product routine per dimension for the instance being run (copied
// from TtnInstance::mp_variant at kernel start; zero = default rule).
__shared__ unsigned char s_mpv[TTN_MAXCHI + 1];
// Tensor-core state of the block when its instance uses the tcgen05
// product: allocated tensor-memory columns, the MMA-completion mbarrier and
// its phase, and the status word a lost MMA is reported to.
__shared__ int s_tc_on;
__shared__ uint32_t s_tc_taddr;
__shared__ uint32_t s_tc_phase;
__shared__ __align__(8) uint64_t s_tc_bar;
__shared__ int* s_tc_status;

// Sub-phase cycle counters (thread 0 of the counting block).
__shared__ unsigned long long s_sub[8];
__device__ __forceinline__ long long sub_start() { return clock64(); }
__device__ __forceinline__ void sub_stop(int idx, long long t0) {
    if (threadIdx.x == 0 && s_count) s_sub[idx] += (unsigned long long)(clock64() - t0);
}

// ---------------------------------------------------------------------------
// teams
// ---------------------------------------------------------------------------
template <int NT_>
struct Solo {
    static constexpr bool wide = false;
    static constexpr int NT = NT_;
    __device__ __forceinline__ int rank() const { return 0; }
    __device__ __forceinline__ int size() const { return 1; }
    __device__ __forceinline__ int tid() const { return threadIdx.x; }
    __device__ __forceinline__ int nthr() const { return NT; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};

struct Clu {
    static constexpr bool wide = true;
    static constexpr int NT = 512;
    int r, n;
    mutable int par;        // parity of the next cross-block exchange buffer
    __device__ __forceinline__ int rank() const { return r; }
    __device__ __forceinline__ int size() const { return n; }
    __device__ __forceinline__ int tid() const { return r * NT + (int)threadIdx.x; }
    __device__ __forceinline__ int nthr() const { return n * NT; }
    __device__ __forceinline__ void sync() const { cg::this_cluster().sync(); }
    // The same shared-memory object in block q of the cluster.
    template <class P>
    __device__ __forceinline__ P* remote(P* p, int q) const { return cg::this_cluster().map_shared_rank(p, q); }
    // Exchange buffers are double-buffered: two uses of one buffer are
    // always separated by another cluster barrier, so a block never
    // overwrites a value another block may still be reading.
    __device__ __forceinline__ int next() const { const int p = par; par ^= 1; return p; }
};

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 cd(double2 a) { return a; }
__device__ __forceinline__ double2 cd(float2 a) { return make_double2(a.x, a.y); }
template <class T> __device__ __forceinline__ T cT(double2 a);
template <> __device__ __forceinline__ double2 cT<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 cT<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconjmul(double2 a, double2 b) {   // conj(a) * b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    double den = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}

// bulk multiply-accumulate in the element type's precision
__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) * b in the element type's precision
__device__ __forceinline__ void cfmaconj(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfmaconj(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(-a.y, b.x, acc.y);
}
template <class T> __device__ __forceinline__ T czero();
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }

// Long sums of complex64 products are accumulated in short blocks whose
// FP32 partials are folded into a compensated running sum (s, c): Knuth's
// TwoSum keeps the rounding error of each fold exactly, so the error of the
// whole sum is that of one block (a few eps) instead of growing with its
// length, at 6 FP32 additions per fold -- while an FP64 accumulator would
// cost 64 FFMA issue slots per add on this part.  complex128 sums are
// plain (c stays unused).
__device__ __forceinline__ void two_sum_into(float& s, float& c, float b) {
    const float t = s + b;
    const float bp = t - s;
    c += (s - (t - bp)) + (b - bp);
    s = t;
}
__device__ __forceinline__ void fold(float2& s, float2& c, float2 b) {
    two_sum_into(s.x, c.x, b.x);
    two_sum_into(s.y, c.y, b.y);
}
__device__ __forceinline__ void fold(double2& s, double2&, double2 b) { s.x += b.x; s.y += b.y; }
__device__ __forceinline__ double2 folded(float2 s, float2 c) { return make_double2((double)s.x + c.x, (double)s.y + c.y); }
__device__ __forceinline__ double2 folded(double2 s, double2) { return s; }

__device__ __forceinline__ double2 warp_sum(double2 v) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ---------------------------------------------------------------------------
// shared scratch
// ---------------------------------------------------------------------------
struct Smem {
    double2 H[(TTN_KMAX + 1) * TTN_KMAX];   // projected matrix, row-major, ld TTN_KMAX
    double2 y[TTN_KMAX + 1];
    double2 u[TTN_KMAX + 1];
    double2 dots[TTN_KMAX + 1];
    double2 red[kMaxWarps * 4];
    double2 bc[4];
    double2 qtau[TTN_MAXCHI];
    int qskip[TTN_MAXCHI];
    double qsign[TTN_MAXCHI];
    int flag;
    // Gram-Schmidt dot products: per-warp partials, block totals
    double2 gsw[kMaxWarps][TTN_KMAX + 1];
    // cross-block exchange (cluster teams)
    double2 xred[2][4];
    int xflag[2];
    double2 qd[2][TTN_MAXCHI];
    double2 xgs[2][TTN_KMAX + 1];
};

// Sum over the blocks of a cluster of the value each block holds at the
// same shared-memory location: lane q of the calling warp reads block q's
// copy and the warp adds them by the xor butterfly, which leaves the same
// bits in every lane, every warp and every block (call with a whole warp;
// the team has at most 32 blocks).
__device__ __forceinline__ double2 gather_sum(const Clu& tm, double2* local) {
    const int lane = threadIdx.x & 31;
    double2 v = lane < tm.size() ? *tm.remote(local, lane) : make_double2(0.0, 0.0);
    return warp_sum(v);
}

// Team-wide sum of one complex value per thread; every thread of the team
// receives the same result.
template <class TM>
__device__ double2 team_sum(double2 v, Smem& sm, const TM& tm) {
    constexpr int W = TM::NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) sm.red[warp] = v;
    __syncthreads();
    if constexpr (!TM::wide) {
        if (warp == 0) {
            double2 w = lane < W ? sm.red[lane] : make_double2(0.0, 0.0);
            w = warp_sum(w);
            if (lane == 0) sm.bc[0] = w;
        }
        __syncthreads();
        double2 r = sm.bc[0];
        __syncthreads();
        return r;
    } else {
        const int p = tm.next();
        if (warp == 0) {
            double2 w = lane < W ? sm.red[lane] : make_double2(0.0, 0.0);
            w = warp_sum(w);
            if (lane == 0) sm.xred[p][0] = w;
        }
        tm.sync();
        return gather_sum(tm, &sm.xred[p][0]);
    }
}

// Four team-wide sums at once (one barrier round); results in sm.bc[0..3].
template <class TM>
__device__ void team_sum4(double2 v[4], Smem& sm, const TM& tm) {
    constexpr int W = TM::NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        v[q] = warp_sum(v[q]);
        if (lane == 0) sm.red[warp * 4 + q] = v[q];
    }
    __syncthreads();
    if constexpr (!TM::wide) {
        if (warp == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                double2 w = lane < W ? sm.red[lane * 4 + q] : make_double2(0.0, 0.0);
                w = warp_sum(w);
                if (lane == 0) sm.bc[q] = w;
            }
        }
        __syncthreads();
    } else {
        const int p = tm.next();
        if (warp == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                double2 w = lane < W ? sm.red[lane * 4 + q] : make_double2(0.0, 0.0);
                w = warp_sum(w);
                if (lane == 0) sm.xred[p][q] = w;
            }
        }
        tm.sync();
        if (warp < 4) {
            const double2 r = gather_sum(tm, &sm.xred[p][warp]);
            if (lane == 0) sm.bc[warp] = r;
        }
        __syncthreads();
    }
}

// One integer decided by the team's first block, seen by every block (the
// stop decisions of the interpreter loop).
template <class TM>
__device__ int team_flag(int v, Smem& sm, const TM& tm) {
    if constexpr (!TM::wide) {
        if (threadIdx.x == 0) sm.flag = v;
        __syncthreads();
        const int r = sm.flag;
        __syncthreads();
        return r;
    } else {
        const int p = tm.next();
        if (threadIdx.x == 0 && tm.rank() == 0) sm.xflag[p] = v;
        tm.sync();
        return *tm.remote(&sm.xflag[p], 0);
    }
}

template <class T, class TM>
__device__ double2 team_dot(const T* a, const T* b, int64_t n, Smem& sm, const TM& tm) {
    T acc = czero<T>(), cmp = czero<T>();
    const int64_t ts = tm.nthr();
    for (int64_t i0 = tm.tid(); i0 < n; i0 += 16 * ts) {
        T blk = czero<T>();
        for (int64_t i = i0, k = 0; k < 16 && i < n; ++k, i += ts) cfmaconj(blk, a[i], b[i]);
        fold(acc, cmp, blk);
    }
    count_flops_t<T>(8.0 * n);
    return team_sum(folded(acc, cmp), sm, tm);
}

// ---------------------------------------------------------------------------
// tensor primitives
// ---------------------------------------------------------------------------
struct Shape {
    int D;
    int d[TTN_MAXD];
    int nset = 1;           // set blocks (multi-set tensors: nset blocks of size() each, back to back)
    __device__ int64_t size() const { int64_t s = 1; for (int j = 0; j < D; ++j) s *= d[j]; return s; }
    __device__ int64_t vlen() const { return size() * nset; }
    __device__ int64_t before(int k) const { int64_t s = 1; for (int j = 0; j < k; ++j) s *= d[j]; return s; }
    __device__ int64_t after(int k) const { int64_t s = 1; for (int j = k + 1; j < D; ++j) s *= d[j]; return s; }
};

// out[l, p, r] (+)= w * sum_m M[p, m] in[l, m, r]   (M: nout x nin, or its
// transpose stored nin x nout when transM).  Generic version: one output
// per thread.
template <class T, class TM>
__device__ void mode_prod_simple(T* out, const T* in, int64_t L, int nin, int nout, int64_t R, const T* M,
                                 bool transM, double2 w, bool accumulate, const TM& tm) {
    const int64_t total = L * nout * R;
    const T wt = cT<T>(w);
    for (int64_t idx = tm.tid(); idx < total; idx += tm.nthr()) {
        const int64_t r = idx % R;
        const int64_t t = idx / R;
        const int p = (int)(t % nout);
        const int64_t l = t / nout;
        const T* src = in + l * nin * R + r;
        T acc = czero<T>();
        if (transM) {
            for (int m = 0; m < nin; ++m) cfma(acc, M[m * nout + p], src[m * R]);
        } else {
            const T* row = M + p * nin;
            for (int m = 0; m < nin; ++m) cfma(acc, row[m], src[m * R]);
        }
        T v = czero<T>();
        cfma(v, wt, acc);
        if (accumulate) { T o = out[idx]; o.x += v.x; o.y += v.y; out[idx] = o; }
        else out[idx] = v;
    }
    tm.sync();
}

// Square mode product with the matrix staged in shared memory and each
// fibre in[l, :, r] held in registers: every thread produces all n outputs
// of its fibre, reading the matrix rows as shared-memory broadcasts.  Two
// outputs are accumulated per pass, so four independent FMA chains hide
// the FMA latency (one pass per output left half of the issue slots idle).
template <class T, int MAXN, class TM>
__device__ void mode_prod_tiled(T* out, const T* in, int64_t L, int n, int64_t R, const T* M, double2 w,
                                bool accumulate, const TM& tm) {
    T* Ms = (T*)dyn_smem;
    for (int i = threadIdx.x; i < n * n; i += TM::NT) Ms[i] = M[i];
    __syncthreads();
    const int64_t F = L * R;
    const T wt = cT<T>(w);
    for (int64_t f = tm.tid(); f < F; f += tm.nthr()) {
        const int64_t l = f / R, r = f - (f / R) * R;
        const T* src = in + l * n * R + r;
        T* dst = out + l * n * R + r;
        T x[MAXN];
#pragma unroll
        for (int m = 0; m < MAXN; ++m) x[m] = (m < n) ? src[m * R] : czero<T>();
        int p = 0;
        for (; p + 1 < n; p += 2) {
            const T* row0 = Ms + p * n;
            const T* row1 = row0 + n;
            T a0 = czero<T>(), a1 = czero<T>();
#pragma unroll
            for (int m = 0; m < MAXN; ++m)
                if (m < n) { cfma(a0, row0[m], x[m]); cfma(a1, row1[m], x[m]); }
            T v0 = czero<T>(), v1 = czero<T>();
            cfma(v0, wt, a0);
            cfma(v1, wt, a1);
            if (accumulate) {
                T o0 = dst[p * R], o1 = dst[(p + 1) * R];
                o0.x += v0.x; o0.y += v0.y; o1.x += v1.x; o1.y += v1.y;
                dst[p * R] = o0; dst[(p + 1) * R] = o1;
            } else {
                dst[p * R] = v0; dst[(p + 1) * R] = v1;
            }
        }
        if (p < n) {
            const T* row = Ms + p * n;
            T acc = czero<T>();
#pragma unroll
            for (int m = 0; m < MAXN; ++m)
                if (m < n) cfma(acc, row[m], x[m]);
            T v = czero<T>();
            cfma(v, wt, acc);
            if (accumulate) { T o = dst[p * R]; o.x += v.x; o.y += v.y; dst[p * R] = o; }
            else dst[p * R] = v;
        }
    }
    tm.sync();
}

// Square mode product for dimensions above the register-fibre limit: the
// transposed matrix Mt[m][p] and a tile of FT fibres Xs[m][f] are staged in
// shared memory; thread (f, pb) accumulates the PB outputs p in
// [pb*PB, pb*PB+PB) of fibre f, reading its fibre value once per m and the
// matrix row segment as a broadcast (PB complex FMAs per shared load of the
// fibre).  Tiles are dealt out to the team's blocks.
template <class T, int PB, class TM>
__device__ void mode_prod_staged(T* out, const T* in, int64_t L, int n, int64_t R, const T* M, double2 w,
                                 bool accumulate, const TM& tm) {
    constexpr int NT = TM::NT;
    constexpr int64_t kBytes = TM::wide ? kStageBytesClu : kStageBytes;
    T* Mt = (T*)dyn_smem;
    for (int i = threadIdx.x; i < n * n; i += NT) {
        const int p = i / n, m = i - p * n;
        Mt[m * n + p] = M[i];
    }
    const int npb = (n + PB - 1) / PB;
    int FT = NT / npb;
    const int64_t cap = (kBytes / (int64_t)sizeof(T) - (int64_t)n * n) / n - 1;
    if (FT > cap) FT = (int)cap;
    const int ld = FT + 1;
    T* Xs = Mt + n * n;
    const int64_t F = L * R;
    const int64_t ntile = (F + FT - 1) / FT;
    const T wt = cT<T>(w);
    const int f = threadIdx.x % FT, pb = threadIdx.x / FT;
    const int p0 = pb * PB;
    const int MS = NT / FT;                          // fibre loads: thread -> (fibre f, m = pb, pb + MS, ...)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t tile = tm.rank(); tile < ntile; tile += tm.size()) {
        const int64_t f0 = tile * FT;
        const int nf = (int)((F - f0) < FT ? (F - f0) : FT);
        __syncthreads();
        if (R == 1) {
            // whole fibres are contiguous rows: warps take fibres, lanes the row
            for (int ff = warp; ff < nf; ff += NT / 32) {
                const T* src = in + (f0 + ff) * n;
                for (int m = lane; m < n; m += 32) Xs[m * ld + ff] = src[m];
            }
        } else if (f < nf && pb < MS) {
            // consecutive threads take consecutive fibres (consecutive r); one
            // division per tile locates the fibre
            const int64_t g = f0 + f, l = g / R, r = g - l * R;
            const T* src = in + l * n * R + r;
            for (int m = pb; m < n; m += MS) Xs[m * ld + f] = src[(int64_t)m * R];
        }
        __syncthreads();
        if (pb < npb && f < nf) {
            T acc[PB];
#pragma unroll
            for (int q = 0; q < PB; ++q) acc[q] = czero<T>();
            for (int m = 0; m < n; ++m) {
                const T x = Xs[m * ld + f];
                const T* mr = Mt + m * n + p0;
#pragma unroll
                for (int q = 0; q < PB; ++q)
                    if (p0 + q < n) cfma(acc[q], mr[q], x);
            }
            const int64_t g = f0 + f, l = g / R, r = g - l * R;
            T* dst = out + l * n * R + r;
#pragma unroll
            for (int q = 0; q < PB; ++q) {
                if (p0 + q >= n) break;
                T v = czero<T>();
                cfma(v, wt, acc[q]);
                if (accumulate) { T o = dst[(p0 + q) * R]; o.x += v.x; o.y += v.y; dst[(p0 + q) * R] = o; }
                else dst[(p0 + q) * R] = v;
            }
        }
    }
    tm.sync();
}

template <class T, class TM>
__device__ void mode_prod(T* out, const T* in, int64_t L, int nin, int nout, int64_t R, const T* M, bool transM,
                          double2 w, bool accumulate, const TM& tm) {
    count_flops_t<T>(8.0 * (double)(L * nout * R) * nin);
    if (transM || nin != nout) {
        mode_prod_simple(out, in, L, nin, nout, R, M, transM, w, accumulate, tm);
        return;
    }
#if TTN_WITH_TC
    if constexpr (sizeof(T) == 8) {
        // tensor cores (3xTF32) where the variant table asks for them and the
        // operands fit the staging area (only in the builds that carry the
        // tensor-core path: a kernel holding tcgen05 code lost the overlap of
        // two co-resident blocks per SM, so the default build has none)
        constexpr int stage = TM::wide ? kStageBytesClu : kStageBytes;
        if (s_mpv[nin] == 2 && s_tc_on && tc_fits(nin, stage)) {
            uint32_t ph = s_tc_phase;
            const int err = tc_mode_prod<TM::NT>((float2*)out, (const float2*)in, L, nin, R, (const float2*)M, w,
                                                 accumulate, dyn_smem, stage, s_tc_taddr, &s_tc_bar, ph, tm.rank(),
                                                 tm.size());
            __syncthreads();
            if (threadIdx.x == 0) {
                s_tc_phase = ph;
                if (err && s_tc_status) atomicExch(s_tc_status, 5);    // TTN_E_TIMEOUT
            }
            tm.sync();
            return;
        }
    }
#endif
    if (nin > (sizeof(T) == 16 ? 16 : 32) || s_mpv[nin] != 0) {
        mode_prod_staged<T, (sizeof(T) == 16 ? 4 : 8)>(out, in, L, nin, R, M, w, accumulate, tm);
        return;
    }
    if (nin <= 2) mode_prod_tiled<T, 2>(out, in, L, nin, R, M, w, accumulate, tm);
    else if (nin <= 4) mode_prod_tiled<T, 4>(out, in, L, nin, R, M, w, accumulate, tm);
    else if (nin <= 8) mode_prod_tiled<T, 8>(out, in, L, nin, R, M, w, accumulate, tm);
    else if (nin <= 12) mode_prod_tiled<T, 12>(out, in, L, nin, R, M, w, accumulate, tm);
    else if (nin <= 16) mode_prod_tiled<T, 16>(out, in, L, nin, R, M, w, accumulate, tm);
    else if (sizeof(T) == 8 && nin <= 24) mode_prod_tiled<T, (sizeof(T) == 8 ? 24 : 16)>(out, in, L, nin, R, M, w, accumulate, tm);
    else if (sizeof(T) == 8) mode_prod_tiled<T, (sizeof(T) == 8 ? 32 : 16)>(out, in, L, nin, R, M, w, accumulate, tm);
}

template <class T, class TM>
__device__ void copy_vec(T* dst, const T* src, int64_t n, const TM& tm) {
    for (int64_t i = tm.tid(); i < n; i += tm.nthr()) dst[i] = src[i];
}

// Chain of mode products of one entry over the modes != skip (skip = -1:
// all modes).  Returns the buffer holding the result (src itself if the
// entry has no factor there).  The last factor is added to `last_out` with
// weight w when last_out != nullptr (written instead of added when
// accumulate_last is false).  Every mode product ends with a team barrier.
template <class T, class TM>
__device__ const T* apply_chain(const T* src, T* t1, T* t2, const Shape& sh, const TtnEntry& e,
                                const TtnSlot* slots, int skip, T* last_out, double2 w, const TM& tm,
                                bool accumulate_last = true) {
    int modes[TTN_MAXD], nf = 0;
    for (int j = 0; j < sh.D; ++j)
        if (j != skip && e.slot[j] >= 0) modes[nf++] = j;
    const T* cur = src;
    for (int f = 0; f < nf; ++f) {
        const int j = modes[f];
        const TtnSlot s = slots[e.slot[j]];
        const T* M = (const T*)s.ptr;
        const int64_t L = sh.before(j), R = sh.after(j);
        const int n = sh.d[j];
        if (f == nf - 1 && last_out) {
            mode_prod(last_out, cur, L, n, n, R, M, false, w, accumulate_last, tm);
            return last_out;
        }
        T* dst = (cur == t1) ? t2 : t1;
        mode_prod(dst, cur, L, n, n, R, M, false, make_double2(1.0, 0.0), false, tm);
        cur = dst;
    }
    return cur;
}

__device__ __forceinline__ int last_factor(const TtnEntry& e, int D) {
    int lm = -1;
    for (int j = 0; j < D; ++j) if (e.slot[j] >= 0) lm = j;
    return lm;
}
__device__ __forceinline__ int n_factors(const TtnEntry& e, int D) {
    int n = 0;
    for (int j = 0; j < D; ++j) n += e.slot[j] >= 0;
    return n;
}

// out = sum_e w_e (x_j M_ej) in   (effective Hamiltonian / bond operator).
// Entries are ordered so that those sharing their last factor (highest mode
// with a matrix, same slot) are adjacent; their partial chains are summed in
// t3 and the shared factor is applied once.
// With sh.nset > 1 (multi-set, paper Sec. II.A) in and out hold nset blocks
// of sh.size() elements; entry e reads block e.src and adds into block
// e.dst, so out is cleared first and every entry accumulates.
template <class T, class TM>
__device__ void heff_apply(T* out, const T* in, T* t1, T* t2, T* t3, const Shape& sh, const TtnEntry* es, int ne,
                           const TtnSlot* slots, const TM& tm) {
    const int64_t S = sh.size();
    const bool multi = sh.nset > 1;
    bool fresh = true;                          // out not written yet: the first term writes it
    if (multi) {
        for (int64_t q = tm.tid(); q < S * sh.nset; q += tm.nthr()) out[q] = czero<T>();
        tm.sync();
        fresh = false;
    }
    int i = 0;
    while (i < ne) {
        const TtnEntry e = es[i];
        const double2 w = make_double2(e.wr, e.wi);
        const int lm = last_factor(e, sh.D);
        const T* ine = multi ? in + (int64_t)e.src * S : in;
        T* oute = multi ? out + (int64_t)e.dst * S : out;
        if (lm < 0) {
            const T wt = cT<T>(w);
            for (int64_t q = tm.tid(); q < S; q += tm.nthr()) {
                T o = fresh ? czero<T>() : oute[q];
                cfma(o, wt, ine[q]);
                oute[q] = o;
            }
            tm.sync();
            fresh = false;
            ++i;
            continue;
        }
        int j = i + 1;
        if (n_factors(e, sh.D) >= 2)
            while (j < ne && last_factor(es[j], sh.D) == lm && es[j].slot[lm] == e.slot[lm] &&
                   n_factors(es[j], sh.D) >= 2 && (!multi || es[j].dst == e.dst)) ++j;
        if (j - i == 1) {
            apply_chain(ine, t1, t2, sh, e, slots, -1, oute, w, tm, !fresh);
            fresh = false;
            i = j;
            continue;
        }
        for (int q = i; q < j; ++q) {
            const TtnEntry eq = es[q];
            const T* inq = multi ? in + (int64_t)eq.src * S : in;
            apply_chain(inq, t1, t2, sh, eq, slots, lm, t3, make_double2(eq.wr, eq.wi), tm, q > i);
        }
        const int n = sh.d[lm];
        mode_prod(oute, (const T*)t3, sh.before(lm), n, n, sh.after(lm), (const T*)slots[e.slot[lm]].ptr, false,
                  make_double2(1.0, 0.0), !fresh, tm);
        fresh = false;
        i = j;
    }
    if (fresh) {                                // no terms: the zero operator
        for (int64_t q = tm.tid(); q < S; q += tm.nthr()) out[q] = czero<T>();
        tm.sync();
    }
}

// G[a, b] += w * sum_{other indices} conj(X[.., a, ..]) Y[.., b, ..]   (index k kept)
// Tiles of X and Y (all chi values of the kept index for OT positions of
// the others) are staged in shared memory; every thread accumulates a 2x2
// block of G, small G are split over groups of positions, and the group
// partials are reduced in a fixed order (deterministic).  A cluster team
// deals the tiles out to its blocks and adds the blocks' partials in rank
// order.
template <class T, class TM>
__device__ void gram_acc(T* G, const T* X, const T* Y, const Shape& sh, int k, double2 w, const TM& tm) {
    constexpr int NT = TM::NT;
    const int chi = sh.d[k];
    const int64_t L = sh.before(k), R = sh.after(k), O = L * R;
    count_flops_t<T>(8.0 * (double)O * chi * chi);
    int OT = (kStageBytes / 2) / (chi * (int)sizeof(T));
    if (OT > 128) OT = 128;
    T* Xs = (T*)dyn_smem;            // [OT][chi]
    T* Ys = Xs + OT * chi;
    const int tn = (chi + 1) / 2, ntile = tn * tn;
    int groups = NT / ntile;
    if (groups < 1) groups = 1;
    if (groups > 8) groups = 8;
    const int tid = threadIdx.x;
    const bool active = tid < ntile * groups || ntile > NT;
    T acc[2][2][2], cmp[2][2][2];                // running sums and their compensations
    const int nrep = (ntile + NT - 1) / NT;      // tiles per thread when chi is large
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) { acc[q][i][j] = czero<T>(); cmp[q][i][j] = czero<T>(); }
    const int g = (ntile >= NT) ? 0 : tid / ntile;
    const int gcount = (ntile >= NT) ? 1 : groups;
    const int64_t ntiles = (O + OT - 1) / OT;
    const int SA = NT / OT, soo = tid % OT, sa = tid / OT;    // staging: thread -> (position, a = sa, sa + SA, ...)
    for (int64_t ti = tm.rank(); ti < ntiles; ti += tm.size()) {
        const int64_t o0 = ti * OT;
        const int nt = (int)((O - o0) < OT ? (O - o0) : OT);
        if (R == 1) {
            const T* xs = X + o0 * chi;
            const T* ys = Y + o0 * chi;
            for (int i = tid; i < nt * chi; i += NT) { Xs[i] = xs[i]; Ys[i] = ys[i]; }
        } else if (soo < nt && sa < SA) {
            // consecutive threads take consecutive positions (consecutive r);
            // one division per tile locates the position
            const int64_t o = o0 + soo, l = o / R, r = o - l * R;
            const int64_t base = l * chi * R + r;
            for (int a = sa; a < chi; a += SA) {
                Xs[soo * chi + a] = X[base + (int64_t)a * R];
                Ys[soo * chi + a] = Y[base + (int64_t)a * R];
            }
        }
        __syncthreads();
        if (active) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (q >= nrep) break;
                const int tile = (ntile >= NT) ? tid + q * NT : tid % ntile;
                if (tile >= ntile) break;
                const int a0 = 2 * (tile / tn), b0 = 2 * (tile % tn);
                const bool a1ok = a0 + 1 < chi, b1ok = b0 + 1 < chi;
                T p00 = czero<T>(), p01 = czero<T>(), p10 = czero<T>(), p11 = czero<T>();
                for (int oo = g; oo < nt; oo += gcount) {
                    const T x0 = Xs[oo * chi + a0];
                    const T x1 = a1ok ? Xs[oo * chi + a0 + 1] : czero<T>();
                    const T y0 = Ys[oo * chi + b0];
                    const T y1 = b1ok ? Ys[oo * chi + b0 + 1] : czero<T>();
                    cfmaconj(p00, x0, y0); cfmaconj(p01, x0, y1);
                    cfmaconj(p10, x1, y0); cfmaconj(p11, x1, y1);
                }
                fold(acc[q][0][0], cmp[q][0][0], p00); fold(acc[q][0][1], cmp[q][0][1], p01);
                fold(acc[q][1][0], cmp[q][1][0], p10); fold(acc[q][1][1], cmp[q][1][1], p11);
            }
        }
        __syncthreads();
    }
    // write partials P[g][a][b] and reduce over g in order
    T* Pp = (T*)dyn_smem;
    if (active) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            if (q >= nrep) break;
            const int tile = (ntile >= NT) ? tid + q * NT : tid % ntile;
            if (tile >= ntile) break;
            const int a0 = 2 * (tile / tn), b0 = 2 * (tile % tn);
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j)
                    if (a0 + i < chi && b0 + j < chi) {
                        T v = acc[q][i][j];
                        v.x += cmp[q][i][j].x;       // (complex128: cmp is zero)
                        v.y += cmp[q][i][j].y;
                        Pp[((int64_t)g * chi + a0 + i) * chi + b0 + j] = v;
                    }
        }
    }
    __syncthreads();
    if constexpr (!TM::wide) {
        for (int ab = tid; ab < chi * chi; ab += NT) {
            double2 sum = make_double2(0.0, 0.0);
            for (int gg = 0; gg < gcount; ++gg) sum = cadd(sum, cd(Pp[(int64_t)gg * chi * chi + ab]));
            G[ab] = cT<T>(cadd(cd(G[ab]), cmul(w, sum)));
        }
        __syncthreads();
    } else {
        // this block's partial in FP64 in the second stage area, then the
        // blocks' partials added in rank order
        double2* Pd = (double2*)(dyn_smem + kStageBytes);
        for (int ab = tid; ab < chi * chi; ab += NT) {
            double2 sum = make_double2(0.0, 0.0);
            for (int gg = 0; gg < gcount; ++gg) sum = cadd(sum, cd(Pp[(int64_t)gg * chi * chi + ab]));
            Pd[ab] = sum;
        }
        tm.sync();
        // thread -> (entry ab, block q): n = team size (a power of two <= 16)
        // consecutive lanes hold the n blocks' partials of one entry and add
        // them by a butterfly confined to their group
        const int nb = tm.size(), per = NT / nb;
        const int q = tid % nb;
        for (int base = tm.rank() * per; base < chi * chi; base += nb * per) {
            const int ab = base + tid / nb;
            double2 v = ab < chi * chi ? tm.remote(Pd, q)[ab] : make_double2(0.0, 0.0);
            for (int o = nb >> 1; o > 0; o >>= 1) {
                v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
                v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
            }
            if (q == 0 && ab < chi * chi) G[ab] = cT<T>(cadd(cd(G[ab]), cmul(w, v)));
        }
        tm.sync();
    }
}

// Environment build: for every output slot, out = Q^dag (sum_e w_e x_{j != keep} M_ej) P
// with P = Q (a single set) or the ket set's tensor (a cross-set
// environment of a multi-set state, paper Sec. II.A).  The chains of all
// entries of one output are summed in ysum first, so each output costs one
// Gram contraction.
template <class T, class TM>
__device__ void env_build(const T* Q, const T* P, T* t1, T* t2, T* ysum, const Shape& sh, int keep,
                          const TtnEntry* es, int ne, const TtnSlot* slots, const TM& tm) {
    const int64_t S = sh.size();
    int i = 0;
    while (i < ne) {
        const int outs = es[i].out;
        int j = i;
        while (j < ne && es[j].out == outs) ++j;
        T* out = (T*)slots[outs].ptr;
        const int n = slots[outs].rows * slots[outs].cols;
        for (int q = tm.tid(); q < n; q += tm.nthr()) out[q] = czero<T>();
        const T* Y;
        if (j - i == 1) {
            const TtnEntry e = es[i];
            Y = apply_chain(P, t1, t2, sh, e, slots, keep, (T*)nullptr, make_double2(1.0, 0.0), tm);
            tm.sync();
            const long long tg = sub_start();
            gram_acc(out, Q, Y, sh, keep, make_double2(e.wr, e.wi), tm);
            sub_stop(3, tg);
        } else {
            for (int q = i; q < j; ++q) {
                const TtnEntry e = es[q];
                const double2 w = make_double2(e.wr, e.wi);
                bool any = false;
                for (int m = 0; m < sh.D; ++m) any |= (m != keep && e.slot[m] >= 0);
                if (!any) {
                    const T wt = cT<T>(w);
                    for (int64_t x = tm.tid(); x < S; x += tm.nthr()) {
                        T o = q > i ? ysum[x] : czero<T>();
                        cfma(o, wt, P[x]);
                        ysum[x] = o;
                    }
                    tm.sync();
                } else {
                    apply_chain(P, t1, t2, sh, e, slots, keep, ysum, w, tm, q > i);
                }
            }
            const long long tg = sub_start();
            gram_acc(out, Q, (const T*)ysum, sh, keep, make_double2(1.0, 0.0), tm);
            sub_stop(3, tg);
        }
        i = j;
    }
}

// out = sum w * M  (slot[0] = -1: w * identity)
template <class T, class TM>
__device__ void combo(const TtnEntry* es, int ne, const TtnSlot* slots, const TM& tm) {
    int prev = -1;
    for (int ei = 0; ei < ne; ++ei) {
        const TtnEntry e = es[ei];
        T* out = (T*)slots[e.out].ptr;
        const int n = slots[e.out].rows;
        if (e.out != prev) {
            for (int i = tm.tid(); i < n * n; i += tm.nthr()) out[i] = czero<T>();
            tm.sync();
            prev = e.out;
        }
        const double2 w = make_double2(e.wr, e.wi);
        const T* M = e.slot[0] >= 0 ? (const T*)slots[e.slot[0]].ptr : nullptr;
        for (int i = tm.tid(); i < n * n; i += tm.nthr()) {
            double2 m = M ? cd(M[i]) : make_double2((i / n == i % n) ? 1.0 : 0.0, 0.0);
            out[i] = cT<T>(cadd(cd(out[i]), cmul(w, m)));
        }
        tm.sync();
    }
}

// ---------------------------------------------------------------------------
// Householder QR of the matricisation with index k as the column index.
// A is overwritten by Q; R (n x n, FP64) is left in Wc's upper triangle with
// signs in sm.qsign.  Rank-deficient columns (remainder norm <= tol ||A||_F)
// get the identity reflector, as in the oracle's definition.
// ---------------------------------------------------------------------------
template <class T, class TM>
__device__ void qr_mode_solo(T* A, const Shape& sh, int k, double2* Wc, double2* Qc, double tol, Smem& sm,
                             const TM& tm) {
    constexpr int NT = TM::NT, NW = NT / 32;
    const int n = sh.d[k];
    const int64_t L = sh.before(k), R = sh.after(k), m = L * R, S = m * n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // gather column-major: Wc[j*m + (l*R + r)] = A[(l*n + j)*R + r]
    double2 part = make_double2(0.0, 0.0);
    for (int64_t idx = threadIdx.x; idx < S; idx += NT) {
        const int64_t j = idx / m, I = idx % m;
        const int64_t l = I / R, r = I % R;
        double2 v = cd(A[(l * n + j) * R + r]);
        Wc[idx] = v;
        part.x += cabs2(v);
    }
    const double thr = tol * sqrt(team_sum(part, sm, tm).x);
    for (int j = 0; j < n; ++j) {
        double2* x = Wc + (int64_t)j * m;
        double2 s = make_double2(0.0, 0.0);
        for (int64_t i = j + threadIdx.x; i < m; i += NT) s.x += cabs2(x[i]);
        const double nrm = sqrt(team_sum(s, sm, tm).x);
        const double2 alpha = x[j];
        if (nrm <= thr) {
            for (int64_t i = j + 1 + threadIdx.x; i < m; i += NT) x[i] = make_double2(0.0, 0.0);
            if (threadIdx.x == 0) { sm.qskip[j] = 1; sm.qtau[j] = make_double2(0.0, 0.0); }
            __syncthreads();
            continue;
        }
        const double beta = alpha.x >= 0.0 ? -nrm : nrm;
        const double2 tau = cscale(csub(make_double2(beta, 0.0), alpha), 1.0 / beta);
        const double2 scl = cdiv(make_double2(1.0, 0.0), csub(alpha, make_double2(beta, 0.0)));
        for (int64_t i = j + 1 + threadIdx.x; i < m; i += NT) x[i] = cmul(x[i], scl);
        __syncthreads();
        if (threadIdx.x == 0) { x[j] = make_double2(beta, 0.0); sm.qskip[j] = 0; sm.qtau[j] = tau; }
        const double2 ctau = make_double2(tau.x, -tau.y);
        count_flops_t<double2>(16.0 * (double)(m - j) * (n - j - 1) + 8.0 * (m - j));
        for (int c = j + 1 + warp; c < n; c += NW) {
            double2* y = Wc + (int64_t)c * m;
            double2 acc = make_double2(0.0, 0.0);
            for (int64_t i = j + lane; i < m; i += 32) {
                double2 v = (i == j) ? make_double2(1.0, 0.0) : x[i];
                cfmaconj(acc, v, y[i]);
            }
            acc = warp_sum(acc);
            const double2 f = cmul(ctau, acc);
            const double2 nf = make_double2(-f.x, -f.y);
            for (int64_t i = j + lane; i < m; i += 32) {
                double2 v = (i == j) ? make_double2(1.0, 0.0) : x[i];
                double2 yi = y[i];
                cfma(yi, v, nf);
                y[i] = yi;
            }
        }
        __syncthreads();
    }
    // Q = H_0 .. H_{n-1} I[:, :n]
    for (int64_t idx = threadIdx.x; idx < S; idx += NT) {
        const int64_t c = idx / m, i = idx % m;
        Qc[idx] = make_double2(i == c ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    for (int j = n - 1; j >= 0; --j) {
        if (sm.qskip[j]) continue;
        const double2 tau = sm.qtau[j];
        const double2* x = Wc + (int64_t)j * m;
        count_flops_t<double2>(16.0 * (double)(m - j) * (n - j));
        for (int c = j + warp; c < n; c += NW) {
            double2* y = Qc + (int64_t)c * m;
            double2 acc = make_double2(0.0, 0.0);
            for (int64_t i = j + lane; i < m; i += 32) {
                double2 v = (i == j) ? make_double2(1.0, 0.0) : x[i];
                cfmaconj(acc, v, y[i]);
            }
            acc = warp_sum(acc);
            const double2 f = cmul(tau, acc);
            const double2 nf = make_double2(-f.x, -f.y);
            for (int64_t i = j + lane; i < m; i += 32) {
                double2 v = (i == j) ? make_double2(1.0, 0.0) : x[i];
                double2 yi = y[i];
                cfma(yi, v, nf);
                y[i] = yi;
            }
        }
        __syncthreads();
    }
    // signs: diag(R) real >= 0
    for (int j = threadIdx.x; j < n; j += NT)
        sm.qsign[j] = (!sm.qskip[j] && Wc[(int64_t)j * m + j].x < 0.0) ? -1.0 : 1.0;
    __syncthreads();
    for (int64_t idx = threadIdx.x; idx < S; idx += NT) {
        const int64_t j = idx / m, I = idx % m;
        const int64_t l = I / R, r = I % R;
        A[(l * n + j) * R + r] = cT<T>(cscale(Qc[idx], sm.qsign[j]));
    }
    __syncthreads();
}

// The same factorisation by a cluster: block b owns a contiguous range of
// the m rows of every column and touches only those (gather, reflector
// scaling, updates, Q accumulation, write-back); per column the team sums
// the remainder norm and exchanges the partial reflector dot products of
// all trailing columns at once.  Reflectors, signs and rank decisions are
// the same as for one block.
template <class T>
__device__ void qr_mode_clu(T* A, const Shape& sh, int k, double2* Wc, double2* Qc, double tol, Smem& sm,
                            const Clu& tm) {
    constexpr int NT = Clu::NT, NW = NT / 32;
    const int n = sh.d[k];
    const int64_t L = sh.before(k), R = sh.after(k), m = L * R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t chunk = (m + tm.size() - 1) / tm.size();
    const int64_t r0 = (int64_t)tm.rank() * chunk < m ? (int64_t)tm.rank() * chunk : m;
    const int64_t r1 = r0 + chunk < m ? r0 + chunk : m;
    const int64_t nr = r1 - r0;
    double2 part = make_double2(0.0, 0.0);
    for (int64_t t = threadIdx.x; t < nr * n; t += NT) {
        const int64_t j = t / nr, I = r0 + (t - (t / nr) * nr);
        const int64_t l = I / R, r = I - (I / R) * R;
        const double2 v = cd(A[(l * n + j) * R + r]);
        Wc[j * m + I] = v;
        part.x += cabs2(v);
    }
    const double thr = tol * sqrt(team_sum(part, sm, tm).x);
    for (int j = 0; j < n; ++j) {
        double2* x = Wc + (int64_t)j * m;
        const int64_t lo = j > r0 ? j : r0;
        // remainder norm and the pivot alpha = x[j] in one exchange (row j's
        // owner contributes alpha; it overwrites x[j] with beta below, so no
        // other block reads x[j] itself)
        double2 d4[4] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0),
                         make_double2(0.0, 0.0)};
        for (int64_t i = lo + threadIdx.x; i < r1; i += NT) d4[0].x += cabs2(x[i]);
        if (threadIdx.x == 0 && j >= r0 && j < r1) d4[1] = x[j];
        team_sum4(d4, sm, tm);
        const double nrm = sqrt(sm.bc[0].x);
        const double2 alpha = sm.bc[1];
        if (nrm <= thr) {
            for (int64_t i = (j + 1 > r0 ? j + 1 : r0) + threadIdx.x; i < r1; i += NT) x[i] = make_double2(0.0, 0.0);
            if (threadIdx.x == 0) { sm.qskip[j] = 1; sm.qtau[j] = make_double2(0.0, 0.0); }
            __syncthreads();
            continue;
        }
        const double beta = alpha.x >= 0.0 ? -nrm : nrm;
        const double2 tau = cscale(csub(make_double2(beta, 0.0), alpha), 1.0 / beta);
        const double2 scl = cdiv(make_double2(1.0, 0.0), csub(alpha, make_double2(beta, 0.0)));
        for (int64_t i = (j + 1 > r0 ? j + 1 : r0) + threadIdx.x; i < r1; i += NT) x[i] = cmul(x[i], scl);
        if (threadIdx.x == 0) { sm.qskip[j] = 0; sm.qtau[j] = tau; }
        __syncthreads();
        if (threadIdx.x == 0 && j >= r0 && j < r1) x[j] = make_double2(beta, 0.0);
        const double2 ctau = make_double2(tau.x, -tau.y);
        count_flops_t<double2>(16.0 * (double)(m - j) * (n - j - 1) + 8.0 * (m - j));
        // partial dots of the reflector with every trailing column over own rows
        const int p = tm.next();
        for (int c = j + 1 + warp; c < n; c += NW) {
            const double2* y = Wc + (int64_t)c * m;
            double2 acc = make_double2(0.0, 0.0);
            for (int64_t i = lo + lane; i < r1; i += 32) {
                const double2 v = (i == j) ? make_double2(1.0, 0.0) : x[i];
                cfmaconj(acc, v, y[i]);
            }
            acc = warp_sum(acc);
            if (lane == 0) sm.qd[p][c] = acc;
        }
        tm.sync();
        for (int c = j + 1 + warp; c < n; c += NW) {
            const double2 acc = gather_sum(tm, &sm.qd[p][c]);
            const double2 f = cmul(ctau, acc);
            const double2 nf = make_double2(-f.x, -f.y);
            double2* y = Wc + (int64_t)c * m;
            for (int64_t i = lo + lane; i < r1; i += 32) {
                const double2 v = (i == j) ? make_double2(1.0, 0.0) : x[i];
                double2 yi = y[i];
                cfma(yi, v, nf);
                y[i] = yi;
            }
        }
        __syncthreads();
    }
    // Q = H_0 .. H_{n-1} I[:, :n], own rows
    for (int64_t t = threadIdx.x; t < nr * n; t += NT) {
        const int64_t c = t / nr, i = r0 + (t - (t / nr) * nr);
        Qc[c * m + i] = make_double2(i == c ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    for (int j = n - 1; j >= 0; --j) {
        if (sm.qskip[j]) continue;
        const double2 tau = sm.qtau[j];
        const double2* x = Wc + (int64_t)j * m;
        const int64_t lo = j > r0 ? j : r0;
        count_flops_t<double2>(16.0 * (double)(m - j) * (n - j));
        const int p = tm.next();
        for (int c = j + warp; c < n; c += NW) {
            const double2* y = Qc + (int64_t)c * m;
            double2 acc = make_double2(0.0, 0.0);
            for (int64_t i = lo + lane; i < r1; i += 32) {
                const double2 v = (i == j) ? make_double2(1.0, 0.0) : x[i];
                cfmaconj(acc, v, y[i]);
            }
            acc = warp_sum(acc);
            if (lane == 0) sm.qd[p][c] = acc;
        }
        tm.sync();
        for (int c = j + warp; c < n; c += NW) {
            const double2 acc = gather_sum(tm, &sm.qd[p][c]);
            const double2 f = cmul(tau, acc);
            const double2 nf = make_double2(-f.x, -f.y);
            double2* y = Qc + (int64_t)c * m;
            for (int64_t i = lo + lane; i < r1; i += 32) {
                const double2 v = (i == j) ? make_double2(1.0, 0.0) : x[i];
                double2 yi = y[i];
                cfma(yi, v, nf);
                y[i] = yi;
            }
        }
        __syncthreads();
    }
    tm.sync();                               // diagonal of R visible to every block
    for (int j = threadIdx.x; j < n; j += NT)
        sm.qsign[j] = (!sm.qskip[j] && Wc[(int64_t)j * m + j].x < 0.0) ? -1.0 : 1.0;
    __syncthreads();
    for (int64_t t = threadIdx.x; t < nr * n; t += NT) {
        const int64_t j = t / nr, I = r0 + (t - (t / nr) * nr);
        const int64_t l = I / R, r = I - (I / R) * R;
        A[(l * n + j) * R + r] = cT<T>(cscale(Qc[j * m + I], sm.qsign[j]));
    }
    tm.sync();
}

template <class T, class TM>
__device__ void qr_mode(T* A, const Shape& sh, int k, double2* Wc, double2* Qc, double tol, Smem& sm, const TM& tm) {
    if constexpr (TM::wide) qr_mode_clu(A, sh, k, Wc, Qc, tol, sm, tm);
    else qr_mode_solo(A, sh, k, Wc, Qc, tol, sm, tm);
}

// R[a][b] of the last QR (a <= b), sign-fixed
__device__ __forceinline__ double2 qr_R(const double2* Wc, int64_t m, int a, int b, const Smem& sm) {
    if (a > b) return make_double2(0.0, 0.0);
    return cscale(Wc[(int64_t)b * m + a], sm.qsign[a]);
}

// ---------------------------------------------------------------------------
// Small projected exponential: sm.y = exp(-i tau H_m) e_0 (warp 0 of every
// block; the blocks of a cluster compute the same values).
// Scaling into s substeps of 1-norm theta <= 4, each summed as a Taylor
// series on the vector (Moler & Van Loan, "Nineteen dubious ways", method 1
// with scaling) with the number of terms k chosen so that theta^(k+1)/(k+1)!
// < 1e-17 (k = 14, 18, 24, 32 for theta <= 1/2, 1, 2, 4); a substep's series
// stops early once the 1-norm bound on the remaining terms is below 1e-18 of
// the partial sum.  The work is
// FP64 (two lanes per SM on this part), so fewer, longer substeps matter:
// 8 nu term evaluations instead of 18 nu for 1-norm nu.  For a tridiagonal
// H only the band is used, for an upper Hessenberg one only j >= i - 1.
// ---------------------------------------------------------------------------
__device__ void small_expm(Smem& sm, int m, double tau, bool band) {
    if ((threadIdx.x >> 5) != 0) return;
    const int i = threadIdx.x & 31;
    double colsum = 0.0;
    if (i < m)
        for (int r = 0; r < m; ++r) colsum += sqrt(cabs2(sm.H[r * TTN_KMAX + i]));
    const double nrm = warp_max(colsum) * fabs(tau);
    if (!(nrm <= 1e5)) {            // not finite or absurdly stiff: report NaN, caller fails
        if (i < m) sm.y[i] = make_double2(NAN, NAN);
        __syncwarp();
        return;
    }
    int s = (int)ceil(nrm / 4.0);
    if (s < 1) s = 1;
    const double theta = nrm / s;
    const int kterms = theta <= 0.5 ? 14 : theta <= 1.0 ? 18 : theta <= 2.0 ? 24 : 32;
    const double h = tau / s;
    double2 y = make_double2(i == 0 ? 1.0 : 0.0, 0.0);
    const int jlo = max(0, i - 1);
    const int jhi = band ? min(m - 1, i + 1) : m - 1;
    for (int step = 0; step < s; ++step) {
        double2 term = y, acc = y;
#pragma unroll 1
        for (int kk = 1; kk <= kterms; ++kk) {
            sm.u[i] = term;
            __syncwarp();
            double2 nt = make_double2(0.0, 0.0);
            if (i < m)
                for (int j = jlo; j <= jhi; ++j) nt = cadd(nt, cmul(sm.H[i * TTN_KMAX + j], sm.u[j]));
            __syncwarp();
            const double f = h / kk;
            term = (i < m) ? make_double2(nt.y * f, -nt.x * f) : make_double2(0.0, 0.0);
            acc = cadd(acc, term);
            // ||t_{k+1}||_1 <= theta / (k+1) ||t_k||_1, so once k >= 2 theta the
            // tail is below the current term; stop when m max|t| <= 1e-18 max|acc|
            // (the same decision in every lane and every block of a cluster)
            if ((kk & 1) == 0 && kk >= 2.0 * theta + 1.0) {
                const double t2 = warp_max(cabs2(term)), a2 = warp_max(cabs2(acc));
                if ((double)m * m * t2 <= 1e-36 * a2) break;
            }
        }
        y = acc;
    }
    if (i < m) sm.y[i] = y;
    __syncwarp();
}

// Hermitian eigen-decomposition A = V diag(A') V^H of an n x n complex matrix
// (FP64, row-major, in place: the diagonal of A holds the eigenvalues on
// return) by the cyclic Jacobi method with the parallel round-robin pair
// ordering: in each round n/2 disjoint (p, q) pairs are rotated at once.
// Each rotation is G = diag(1, e^{-i phi}) times the real rotation that
// annihilates the now real off-diagonal element (Golub & Van Loan, Sec. 8.5).
// The rotation parameters of a round are computed by every block (in its
// own shared memory); the rotations themselves are dealt out to the team.
template <class TM>
__device__ __noinline__ void jacobi_eigh(double2* A, double2* Vm, int n, Smem& sm, const TM& tm) {
    constexpr int NT = TM::NT;
    const int tid = threadIdx.x;
    for (int i = tm.tid(); i < n * n; i += tm.nthr()) Vm[i] = make_double2(i / n == i % n ? 1.0 : 0.0, 0.0);
    const int nn = (n + 1) & ~1;
    const int npair = nn / 2;
    double* rc = (double*)dyn_smem;
    double* rs = rc + npair;
    double2* ph = (double2*)(rs + npair);
    int* pp = (int*)(ph + npair);
    int* pq = pp + npair;
    tm.sync();
    for (int sweep = 0; sweep < 60; ++sweep) {
        double2 part = make_double2(0.0, 0.0);
        for (int i = tm.tid(); i < n * n; i += tm.nthr()) {
            const int r = i / n, c = i - r * n;
            if (r != c) part.x += cabs2(A[i]);
            else part.y += A[i].x * A[i].x;
        }
        const double2 nrm = team_sum(part, sm, tm);
        if (nrm.x <= 1e-30 * (nrm.x + nrm.y) || nrm.x == 0.0) break;
        for (int rnd = 0; rnd < nn - 1; ++rnd) {
            for (int i = tid; i < npair; i += NT) {
                const int a = (i == 0) ? 0 : ((i - 1 + rnd) % (nn - 1)) + 1;
                const int jj = nn - 1 - i;
                const int b = ((jj - 1 + rnd) % (nn - 1)) + 1;
                const int p = min(a, b), q = max(a, b);
                double c = 1.0, sn = 0.0;
                double2 e = make_double2(1.0, 0.0);
                if (q < n) {
                    const double2 apq = A[p * n + q];
                    const double r = sqrt(cabs2(apq));
                    if (r > 1e-300) {
                        const double theta = (A[q * n + q].x - A[p * n + p].x) / (2.0 * r);
                        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        sn = t * c;
                        e = make_double2(apq.x / r, -apq.y / r);          // e^{-i phi}
                    }
                }
                rc[i] = c; rs[i] = sn; ph[i] = e; pp[i] = p; pq[i] = q;
            }
            __syncthreads();
            for (int idx = tm.tid(); idx < npair * n; idx += tm.nthr()) {      // columns of A and V
                const int i = idx / n, row = idx - (idx / n) * n;
                const int p = pp[i], q = pq[i];
                if (q >= n || rs[i] == 0.0) continue;
                const double c = rc[i], sn = rs[i];
                const double2 e = ph[i];
                double2 ap = A[row * n + p], aq = cmul(e, A[row * n + q]);
                A[row * n + p] = make_double2(c * ap.x - sn * aq.x, c * ap.y - sn * aq.y);
                A[row * n + q] = make_double2(sn * ap.x + c * aq.x, sn * ap.y + c * aq.y);
                ap = Vm[row * n + p]; aq = cmul(e, Vm[row * n + q]);
                Vm[row * n + p] = make_double2(c * ap.x - sn * aq.x, c * ap.y - sn * aq.y);
                Vm[row * n + q] = make_double2(sn * ap.x + c * aq.x, sn * ap.y + c * aq.y);
            }
            tm.sync();
            for (int idx = tm.tid(); idx < npair * n; idx += tm.nthr()) {      // rows of A
                const int i = idx / n, col = idx - (idx / n) * n;
                const int p = pp[i], q = pq[i];
                if (q >= n || rs[i] == 0.0) continue;
                const double c = rc[i], sn = rs[i];
                const double2 ec = make_double2(ph[i].x, -ph[i].y);     // e^{+i phi}
                const double2 ap = A[p * n + col], aq = cmul(ec, A[q * n + col]);
                A[p * n + col] = make_double2(c * ap.x - sn * aq.x, c * ap.y - sn * aq.y);
                A[q * n + col] = make_double2(sn * ap.x + c * aq.x, sn * ap.y + c * aq.y);
            }
            tm.sync();
        }
    }
}

// Lowest Ritz pair of the m x m Hermitian tridiagonal Lanczos matrix in
// sm.H: eigen-decomposition by cyclic Jacobi in the block's own stage
// buffer (every block of a team does the same), eigenvector to
// sm.y[0..m), eigenvalue to sm.u[0].x.
template <int NT>
__device__ void lowest_ritz(Smem& sm, int m) {
    double2* T = (double2*)(dyn_smem + 16384);
    double2* Vm = (double2*)(dyn_smem + 32768);
    for (int i = threadIdx.x; i < m * m; i += NT) {
        const int r = i / m, c = i - (i / m) * m;
        T[i] = sm.H[r * TTN_KMAX + c];
    }
    __syncthreads();
    jacobi_eigh(T, Vm, m, sm, Solo<NT>());
    if (threadIdx.x == 0) {
        int imin = 0;
        for (int i = 1; i < m; ++i)
            if (T[i * m + i].x < T[imin * m + imin].x) imin = i;
        for (int i = 0; i < m; ++i) sm.y[i] = Vm[i * m + imin];
        sm.u[0] = make_double2(T[imin * m + imin].x, 0.0);
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Krylov exponential x <- exp(-i tau Hop) x (Lanczos when herm, Arnoldi
// otherwise; two classical Gram-Schmidt passes against the whole basis).
// The basis V is kept in the bulk type TB; x (node tensor or bond matrix) in
// the state type TS.  The result is assembled as
//     x_new = y_0 x + ||x|| sum_{i>=1} y_i V_i
// so that the leading term keeps the state's precision.
// Stops on Saad's estimate h_{m+1,m} |e_m^T exp(-i tau H_m) e_1| <= tol.
// Returns 1 when converged (x updated), 0 when kmax was reached, -1 on a
// non-finite norm.
// ---------------------------------------------------------------------------
template <class TS, class TB, class TM>
__device__ int krylov_once(TS* x, const Shape& sh, const TtnEntry* es, int ne, const TtnSlot* slots, double tau,
                           int herm, double tol, int kmax, TB* V, int64_t smax, TB* t1, TB* t2, TB* t3, Smem& sm,
                           const TM& tm, int ground = 0) {
    double logbound = 0.0;          // log(|tau|^m prod h_{i+1,i} / m!)
    const int64_t S = sh.vlen();    // all set blocks form one vector
    const int64_t t0 = tm.tid(), ts = tm.nthr();
    double2 nb = make_double2(0.0, 0.0);
    for (int64_t i = t0; i < S; i += ts) nb.x += cabs2(cd(x[i]));
    const double beta0 = sqrt(team_sum(nb, sm, tm).x);
    if (beta0 == 0.0) return 1;
    if (!isfinite(beta0)) return -1;
    for (int i = threadIdx.x; i < (TTN_KMAX + 1) * TTN_KMAX; i += TM::NT) sm.H[i] = make_double2(0.0, 0.0);
    {
        const double inv = 1.0 / beta0;
        for (int64_t i = t0; i < S; i += ts) V[i] = cT<TB>(cscale(cd(x[i]), inv));
    }
    tm.sync();
    for (int j = 0; j < kmax; ++j) {
        TB* vj = V + (int64_t)j * smax;
        TB* w = V + (int64_t)(j + 1) * smax;
        const long long th = sub_start();
        heff_apply(w, vj, t1, t2, t3, sh, es, ne, slots, tm);
        sub_stop(0, th);
        const long long tgs = sub_start();
        for (int pass = 0; pass < 2; ++pass) {
            // dots <V_i, w> for i <= j: four at a time over the elements,
            // per-warp partials kept in shared memory, then one reduction
            // (one cluster exchange) for all of them
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            constexpr int W = TM::NT / 32;
            for (int i0 = 0; i0 <= j; i0 += 4) {
                const int nb = (j + 1 - i0) < 4 ? (j + 1 - i0) : 4;
                TB acc[4] = {czero<TB>(), czero<TB>(), czero<TB>(), czero<TB>()};
                TB cmp[4] = {czero<TB>(), czero<TB>(), czero<TB>(), czero<TB>()};
                for (int64_t e0 = t0; e0 < S; e0 += 16 * ts) {
                    TB blk[4] = {czero<TB>(), czero<TB>(), czero<TB>(), czero<TB>()};
                    for (int64_t e = e0, k = 0; k < 16 && e < S; ++k, e += ts) {
                        const TB we = w[e];
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (q < nb) cfmaconj(blk[q], V[(int64_t)(i0 + q) * smax + e], we);
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) fold(acc[q], cmp[q], blk[q]);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const double2 d = warp_sum(folded(acc[q], cmp[q]));
                    if (lane == 0 && q < nb) sm.gsw[warp][i0 + q] = d;
                }
            }
            __syncthreads();
            if constexpr (!TM::wide) {
                for (int i = warp; i <= j; i += W) {
                    double2 v = lane < W ? sm.gsw[lane][i] : make_double2(0.0, 0.0);
                    v = warp_sum(v);
                    if (lane == 0) {
                        sm.dots[i] = v;
                        sm.H[i * TTN_KMAX + j] = cadd(sm.H[i * TTN_KMAX + j], v);
                    }
                }
            } else {
                const int p = tm.next();
                for (int i = warp; i <= j; i += W) {
                    double2 v = lane < W ? sm.gsw[lane][i] : make_double2(0.0, 0.0);
                    v = warp_sum(v);
                    if (lane == 0) sm.xgs[p][i] = v;
                }
                tm.sync();
                for (int i = warp; i <= j; i += W) {
                    const double2 v = gather_sum(tm, &sm.xgs[p][i]);
                    if (lane == 0) {
                        sm.dots[i] = v;
                        sm.H[i * TTN_KMAX + j] = cadd(sm.H[i * TTN_KMAX + j], v);
                    }
                }
            }
            __syncthreads();
            count_flops_t<TB>(16.0 * (double)S * (j + 1));
            int64_t e = t0;
            for (; e + ts < S; e += 2 * ts) {
                TB a0 = w[e], a1 = w[e + ts];
                for (int i = 0; i <= j; ++i) {
                    const double2 h = sm.dots[i];
                    const TB nh = cT<TB>(make_double2(-h.x, -h.y));
                    const TB* Vi = V + (int64_t)i * smax + e;
                    cfma(a0, nh, Vi[0]);
                    cfma(a1, nh, Vi[ts]);
                }
                w[e] = a0;
                w[e + ts] = a1;
            }
            if (e < S) {
                TB acc = w[e];
                for (int i = 0; i <= j; ++i) {
                    const double2 h = sm.dots[i];
                    cfma(acc, cT<TB>(make_double2(-h.x, -h.y)), V[(int64_t)i * smax + e]);
                }
                w[e] = acc;
            }
            tm.sync();
        }
        if (herm && threadIdx.x == 0) {
            sm.H[j * TTN_KMAX + j].y = 0.0;
            for (int i = 0; i + 1 < j; ++i) sm.H[i * TTN_KMAX + j] = make_double2(0.0, 0.0);
            if (j > 0) sm.H[(j - 1) * TTN_KMAX + j] = sm.H[j * TTN_KMAX + (j - 1)];
        }
        TB nwt = czero<TB>(), nwc = czero<TB>();
        for (int64_t e0 = t0; e0 < S; e0 += 16 * ts) {
            TB blk = czero<TB>();
            for (int64_t e = e0, k = 0; k < 16 && e < S; ++k, e += ts) cfmaconj(blk, w[e], w[e]);
            fold(nwt, nwc, blk);
        }
        const double hnext = sqrt(team_sum(folded(nwt, nwc), sm, tm).x);
        if (threadIdx.x == 0) sm.H[(j + 1) * TTN_KMAX + j] = make_double2(hnext, 0.0);
        __syncthreads();
        sub_stop(1, tgs);
        const int mm = j + 1;
        if (!isfinite(hnext)) return -1;
        // For a Hermitian tridiagonal H_m, |e_m^T exp(-i tau H_m) e_1| <= |tau|^(m-1)
        // prod_{i<m-1} h_{i+1,i} / (m-1)!, so h_{m+1,m} times that bounds Saad's
        // estimate; the small exponential is evaluated only once this bound is
        // within 1e4 of the tolerance (always at kmax and on breakdown).
        logbound += log(fmax(hnext, 1e-300)) + log(fabs(tau) + 1e-300) - log((double)mm);
        const bool near = ground ? ((j & 1) == 1 || j == kmax - 1 || hnext == 0.0)
                                 : (logbound <= log(1e4 * tol) || j == kmax - 1 || hnext == 0.0 || (j & 3) == 3);
        if (!near) {
            const double inv = 1.0 / hnext;
            for (int64_t e = t0; e < S; e += ts) w[e] = cT<TB>(cscale(cd(w[e]), inv));
            tm.sync();
            continue;
        }
        if (ground) {
            // lowest Ritz pair; Lanczos residual |h_{m+1,m} y_m| against tol * max(1, |theta|)
            lowest_ritz<TM::NT>(sm, mm);
            const double theta = sm.u[0].x;
            const double res = hnext * sqrt(cabs2(sm.y[j]));
            if (!isfinite(res) || !isfinite(theta)) return -1;
            const bool conv = res <= tol * fmax(1.0, fabs(theta)) || hnext == 0.0;
            if (conv || j == kmax - 1) {
                // x <- sum_i y_i V_i with V_0 = x / beta0 taken from x itself, then renormalised
                const double2 y0 = cscale(sm.y[0], 1.0 / beta0);
                count_flops_t<TB>(8.0 * (double)S * mm);
                for (int64_t e = t0; e < S; e += ts) {
                    TB acc = czero<TB>();
                    for (int i = 1; i < mm; ++i) cfma(acc, cT<TB>(sm.y[i]), V[(int64_t)i * smax + e]);
                    x[e] = cT<TS>(cadd(cmul(y0, cd(x[e])), cd(acc)));
                }
                tm.sync();
                double2 nx = make_double2(0.0, 0.0);
                for (int64_t e = t0; e < S; e += ts) nx.x += cabs2(cd(x[e]));
                const double inv = 1.0 / sqrt(team_sum(nx, sm, tm).x);
                for (int64_t e = t0; e < S; e += ts) x[e] = cT<TS>(cscale(cd(x[e]), inv));
                tm.sync();
                return conv ? 1 : 0;
            }
            const double inv = 1.0 / hnext;
            for (int64_t e = t0; e < S; e += ts) w[e] = cT<TB>(cscale(cd(w[e]), inv));
            tm.sync();
            continue;
        }
        const long long te = sub_start();
        small_expm(sm, mm, tau, herm != 0);
        __syncthreads();
        sub_stop(2, te);
        const double err = hnext * sqrt(cabs2(sm.y[j]));
        if (!isfinite(err)) return -1;
        if (err <= tol || hnext == 0.0) {
            const double2 y0 = sm.y[0];
            count_flops_t<TB>(8.0 * (double)S * mm);
            for (int64_t e = t0; e < S; e += ts) {
                TB acc = czero<TB>();
                for (int i = 1; i < mm; ++i) cfma(acc, cT<TB>(sm.y[i]), V[(int64_t)i * smax + e]);
                x[e] = cT<TS>(cadd(cmul(y0, cd(x[e])), cscale(cd(acc), beta0)));
            }
            tm.sync();
            return 1;
        }
        const double inv = 1.0 / hnext;
        for (int64_t e = t0; e < S; e += ts) w[e] = cT<TB>(cscale(cd(w[e]), inv));   // (kept exact in FP64 mode)
        tm.sync();
    }
    return 0;
}

template <class TS, class TB, class TM>
__device__ int krylov_expm(TS* x, const Shape& sh, const TtnEntry* es, int ne, const TtnSlot* slots, double tau,
                           int herm, double tol, int kmax, TB* V, int64_t smax, TB* t1, TB* t2, TB* t3, Smem& sm,
                           const TM& tm) {
    // substeps: halve the interval whenever kmax is reached (at most 2^12 pieces)
    int nsub = 1, done = 0;
    while (done < nsub) {
        const int r = krylov_once(x, sh, es, ne, slots, tau / nsub, herm, tol, kmax, V, smax, t1, t2, t3, sm, tm);
        if (r < 0) return 0;
        if (r > 0) {
            ++done;
        } else {
            if (nsub >= (1 << 12)) return 0;
            nsub *= 2; done *= 2;
        }
    }
    return 1;
}

// Lowest eigenpair of a Hermitian H_eff by restarted Lanczos (restart from
// the current Ritz vector after kmax steps).  Returns 1 and the eigenvalue
// on convergence, 0 otherwise.
template <class TS, class TB, class TM>
__device__ int krylov_ground(TS* x, const Shape& sh, const TtnEntry* es, int ne, const TtnSlot* slots, double tol,
                             int kmax, TB* V, int64_t smax, TB* t1, TB* t2, TB* t3, Smem& sm, double* theta,
                             const TM& tm) {
    for (int r = 0; r < 200; ++r) {
        const int s = krylov_once(x, sh, es, ne, slots, 0.0, 1, tol, kmax, V, smax, t1, t2, t3, sm, tm, 1);
        if (s < 0) return 0;
        if (s > 0) {
            *theta = sm.u[0].x;
            return 1;
        }
    }
    return 0;
}

template <class TB, class TS, class TM>
__device__ const TB* as_bulk(const TS* a, TB* buf, int64_t n, const TM& tm) {
    if (sizeof(TS) == sizeof(TB)) return (const TB*)a;
    const long long t0 = sub_start();
    for (int64_t i = tm.tid(); i < n; i += tm.nthr()) buf[i] = cT<TB>(cd(a[i]));
    tm.sync();
    sub_stop(4, t0);
    return buf;
}

// C = op(A) * B for small dense FP64 matrices (row-major): A is m x k (or
// k x m when adjA, then conjugate-transposed), B is k x n.
template <class TM>
__device__ void small_gemm(double2* C, const double2* A, const double2* B, int m, int k, int n, bool adjA,
                           const TM& tm) {
    for (int idx = tm.tid(); idx < m * n; idx += tm.nthr()) {
        const int i = idx / n, j = idx - (idx / n) * n;
        double2 acc = make_double2(0.0, 0.0);
        for (int l = 0; l < k; ++l) {
            const double2 a = adjA ? make_double2(A[l * m + i].x, -A[l * m + i].y) : A[i * k + l];
            acc = cadd(acc, cmul(a, B[l * n + j]));
        }
        C[idx] = acc;
    }
    count_flops_t<double2>(8.0 * m * k * n);
    tm.sync();
}

// ---------------------------------------------------------------------------
// Subspace expansion (paper Sec. II.D).
// ---------------------------------------------------------------------------
// Test the bond to child c = children(z)[k] for new single-particle
// functions (the centre is at z).  With X_a the child's up channel a applied
// at the two-site level to A^c, W~_a = sum_b w_ab D_b A^z the matching down
// channels applied to A^z, P_c = A^c A^c^dag and P_S the projector on the
// child's single-hole functions (QR of A^z along k),
//     Y = (1 - P_c) G (1 - P_S) = X' W'^T,  Y Y^dag = X' C X'^dag,
// with X' = (1 - P_c) X, W' = (1 - Q_S Q_S^dag) W~, C = W'^T conj W'.  The
// dominant eigenvectors of Y Y^dag are found in span X': with
// E = X'^dag X' = V L V^dag and F = V L^{-1/2} (numerically nonzero part),
// T = F^dag E C E F is Hermitian and its eigenvector w gives u = X' F w.
template <class TS, class TB, class TM>
__device__ __noinline__ void spawn_op(const TtnOp* opg, const TtnInstance* ing, Smem& sm, TB* V, int64_t smax, TB* t1,
                                      TB* t2, double2* Wc, double2* Qc, const TM& tm) {
    // The op and the instance are read from global memory: a reference to
    // the caller's register copies would force those copies into local
    // memory for the whole kernel.
    const TtnOp& op = *opg;
    const TtnInstance& in = *ing;
    const int t0 = tm.tid(), ts = tm.nthr();
    Shape shz, shc;
    shz.D = op.D; shc.D = op.Dc;
    for (int j = 0; j < TTN_MAXD; ++j) {
        shz.d[j] = j < op.D ? op.dims[j] : 1;
        shc.d[j] = j < op.Dc ? op.dimsc[j] : 1;
    }
    const int k = op.k;
    const int chi = shz.d[k];
    const int64_t Sz = shz.size(), Sc = shc.size();
    const int NJ = (int)(Sc / chi), NT = (int)(Sz / chi);
    int cap = min(in.chi_max, min(NJ, NT)) - chi;
    if (cap <= 0 || in.spawn_eps <= 0.0) return;
    if (cap > TTN_SPAWN_MAX_NEW) cap = TTN_SPAWN_MAX_NEW;
    // distinct non-identity up channels among the bond terms
    const TtnEntry* eb = in.entries + op.e2;
    int ids[TTN_SPAWN_MAX_CHANNELS];
    int A = 0;
    bool space = true;
    for (int i = 0; i < op.ne2; ++i) {
        const int a = eb[i].slot[0];
        if (a < 0) continue;
        bool seen = false;
        for (int q = 0; q < A; ++q) seen |= ids[q] == a;
        if (!seen) {
            if (A == TTN_SPAWN_MAX_CHANNELS) { space = false; break; }
            ids[A++] = a;
        }
    }
    const int K = A * chi;
    if (!space || K > in.spawn_kmax) {          // the bond cannot be tested: report, do not skip
        if (threadIdx.x == 0 && tm.rank() == 0) atomicExch(in.status, TTN_STATUS_SPAWN_SPACE);
        tm.sync();
        return;
    }
    if (A == 0) return;
    const TtnSlot* slots = in.slots;
    TB* Mc = V;
    TB* Mz = V + smax;
    TB* X = V + 2 * smax;                       // A buffers of Sc
    TB* Wt = V + (2 + A) * smax;                // A buffers of Sz
    TB* Wb = V + (2 + 2 * A) * smax;
    TB* Qsc = V + (3 + 2 * A) * smax;
    TB* g = V + (4 + 2 * A) * smax;             // chi x chi scratch
    double2* ws = (double2*)in.spawn_ws;
    double2* Acopy = ws;
    double2* E = ws + smax;
    double2* Cm = E + (int64_t)K * K;
    double2* T = Cm + (int64_t)K * K;
    double2* VE = T + (int64_t)K * K;
    double2* WT = VE + (int64_t)K * K;
    double2* P1 = WT + (int64_t)K * K;
    {
        const TS* Ac = (const TS*)op.c;
        const TS* Az = (const TS*)op.a;
        for (int64_t i = t0; i < Sc; i += ts) Mc[i] = cT<TB>(cd(Ac[i]));
        for (int64_t i = t0; i < Sz; i += ts) { Mz[i] = cT<TB>(cd(Az[i])); Acopy[i] = cd(Az[i]); }
        tm.sync();
    }
    const int lastc = shc.D - 1;
    // X_a = (1 - Mc Mc^dag) U_a Mc
    for (int a = 0; a < A; ++a) {
        TB* Xa = X + a * smax;
        for (int64_t i = t0; i < Sc; i += ts) Xa[i] = czero<TB>();
        tm.sync();
        const TtnEntry* eu = in.entries + op.e0;
        for (int i = 0; i < op.ne; ++i) {
            const TtnEntry e = eu[i];
            if (e.out != ids[a]) continue;
            bool any = false;
            for (int m = 0; m < shc.D; ++m) any |= (m != lastc && e.slot[m] >= 0);
            if (!any) {
                const TB wt = cT<TB>(make_double2(e.wr, e.wi));
                for (int64_t x = t0; x < Sc; x += ts) { TB o = Xa[x]; cfma(o, wt, Mc[x]); Xa[x] = o; }
                tm.sync();
            } else {
                apply_chain((const TB*)Mc, t1, t2, shc, e, slots, lastc, Xa, make_double2(e.wr, e.wi), tm);
            }
        }
        for (int i = t0; i < chi * chi; i += ts) g[i] = czero<TB>();
        tm.sync();
        gram_acc(g, (const TB*)Mc, (const TB*)Xa, shc, lastc, make_double2(1.0, 0.0), tm);
        mode_prod(Xa, (const TB*)Mc, shc.before(lastc), chi, chi, (int64_t)1, (const TB*)g, true,
                  make_double2(-1.0, 0.0), true, tm);
    }
    // W~_a = sum_b w_ab D_b Mz
    for (int a = 0; a < A; ++a) {
        TB* Wa = Wt + a * smax;
        for (int64_t i = t0; i < Sz; i += ts) Wa[i] = czero<TB>();
        tm.sync();
        for (int i = 0; i < op.ne2; ++i) {
            const TtnEntry tb = eb[i];
            if (tb.slot[0] != ids[a]) continue;
            const int bsl = tb.slot[1];
            const TB* src = Mz;
            if (bsl >= 0) {
                for (int64_t x = t0; x < Sz; x += ts) Wb[x] = czero<TB>();
                tm.sync();
                const TtnEntry* ed = in.entries + op.e1;
                for (int q = 0; q < op.ne1; ++q) {
                    const TtnEntry e = ed[q];
                    if (e.out != bsl) continue;
                    bool any = false;
                    for (int m = 0; m < shz.D; ++m) any |= (m != k && e.slot[m] >= 0);
                    if (!any) {
                        const TB wt = cT<TB>(make_double2(e.wr, e.wi));
                        for (int64_t x = t0; x < Sz; x += ts) { TB o = Wb[x]; cfma(o, wt, Mz[x]); Wb[x] = o; }
                        tm.sync();
                    } else {
                        apply_chain((const TB*)Mz, t1, t2, shz, e, slots, k, Wb, make_double2(e.wr, e.wi), tm);
                    }
                }
                src = Wb;
            }
            const TB wt = cT<TB>(make_double2(tb.wr, tb.wi));
            for (int64_t x = t0; x < Sz; x += ts) { TB o = Wa[x]; cfma(o, wt, src[x]); Wa[x] = o; }
            tm.sync();
        }
    }
    // single-hole functions: Q of A^z along k (FP64)
    qr_mode(Acopy, shz, k, Wc, Qc, in.qtol, sm, tm);
    for (int64_t i = t0; i < Sz; i += ts) Qsc[i] = cT<TB>(Acopy[i]);
    tm.sync();
    // W'_a = (1 - Qs Qs^dag) W~_a   (G (1 - P_S) = X (W'^T) with P_S acting on rows of G)
    for (int a = 0; a < A; ++a) {
        TB* Wa = Wt + a * smax;
        for (int i = t0; i < chi * chi; i += ts) g[i] = czero<TB>();
        tm.sync();
        gram_acc(g, (const TB*)Qsc, (const TB*)Wa, shz, k, make_double2(1.0, 0.0), tm);
        mode_prod(Wa, (const TB*)Qsc, shz.before(k), chi, chi, shz.after(k), (const TB*)g, true,
                  make_double2(-1.0, 0.0), true, tm);
    }
    // E = X'^dag X', C = conj(W'^dag W')   (K x K, FP64)
    for (int a = 0; a < A; ++a)
        for (int b = 0; b < A; ++b) {
            for (int i = t0; i < chi * chi; i += ts) g[i] = czero<TB>();
            tm.sync();
            gram_acc(g, (const TB*)(X + a * smax), (const TB*)(X + b * smax), shc, lastc, make_double2(1.0, 0.0), tm);
            for (int i = t0; i < chi * chi; i += ts)
                E[(int64_t)(a * chi + i / chi) * K + b * chi + i % chi] = cd(g[i]);
            tm.sync();
            for (int i = t0; i < chi * chi; i += ts) g[i] = czero<TB>();
            tm.sync();
            gram_acc(g, (const TB*)(Wt + a * smax), (const TB*)(Wt + b * smax), shz, k, make_double2(1.0, 0.0), tm);
            for (int i = t0; i < chi * chi; i += ts) {
                const double2 v = cd(g[i]);
                Cm[(int64_t)(a * chi + i / chi) * K + b * chi + i % chi] = make_double2(v.x, -v.y);
            }
            tm.sync();
        }
    // trace(Y Y^dag) = trace(C E) bounds every eigenvalue
    const double thr = (in.spawn_eps / in.spawn_dt) * (in.spawn_eps / in.spawn_dt);
    {
        double2 part = make_double2(0.0, 0.0);
        for (int64_t idx = t0; idx < (int64_t)K * K; idx += ts) {
            const int i = (int)(idx / K), j = (int)(idx % K);
            part = cadd(part, cmul(Cm[(int64_t)i * K + j], E[(int64_t)j * K + i]));
        }
        const double tr = team_sum(part, sm, tm).x;
        if (!(tr >= thr)) return;
    }
    // E = V L V^dag; F = V L^{-1/2} on the numerically nonzero part (stored in P1, K x r)
    for (int64_t i = t0; i < (int64_t)K * K; i += ts) T[i] = E[i];
    tm.sync();
    jacobi_eigh(T, VE, K, sm, tm);
    double lmax = 0.0;
    for (int i = 0; i < K; ++i) lmax = fmax(lmax, T[(int64_t)i * K + i].x);
    const double ltol = lmax * (sizeof(TB) == 16 ? 1e-13 : 1e-7);
    int r = 0;
    int* keep = (int*)(dyn_smem + 32768);
    if (threadIdx.x == 0)
        for (int i = 0; i < K; ++i)
            if (T[(int64_t)i * K + i].x > ltol && lmax > 0.0) keep[r++] = i;
    if (threadIdx.x == 0) sm.flag = r;
    __syncthreads();
    r = sm.flag;
    __syncthreads();
    if (r == 0) return;
    for (int64_t idx = t0; idx < (int64_t)K * r; idx += ts) {
        const int i = (int)(idx / r), j = (int)(idx % r);
        const int kj = keep[j];
        P1[idx] = cscale(VE[(int64_t)i * K + kj], 1.0 / sqrt(T[(int64_t)kj * K + kj].x));
    }
    tm.sync();
    // T = F^dag E C E F  (r x r):  WT = E F (K x r), VE = C WT, T = WT^dag VE
    small_gemm(WT, E, P1, K, K, r, false, tm);
    small_gemm(VE, Cm, WT, K, K, r, false, tm);
    small_gemm(T, WT, VE, r, K, r, true, tm);
    jacobi_eigh(T, Cm, r, sm, tm);                 // eigenvectors of T in Cm (r x r)
    // accept eigenvalues >= thr, largest first
    int* order = keep + TTN_SPAWN_MAX_K;
    if (threadIdx.x == 0) {
        int cnt = 0;
        for (int i = 0; i < r; ++i) order[cnt++] = i;
        for (int i = 0; i < cnt; ++i)
            for (int j = i + 1; j < cnt; ++j)
                if (T[(int64_t)order[j] * r + order[j]].x > T[(int64_t)order[i] * r + order[i]].x) {
                    const int tmp = order[i]; order[i] = order[j]; order[j] = tmp;
                }
        // complex64 contractions leave noise of ~1e-7 of the largest eigenvalue
        // in T: with a complex64 bulk only eigenvalues above 1e-6 of the
        // largest are taken as resolved (complex128: the oracle's rule alone)
        const double tfloor = sizeof(TB) == 16 ? 0.0 : 1e-6 * (cnt > 0 ? T[(int64_t)order[0] * r + order[0]].x : 0.0);
        int p = 0;
        while (p < cnt && p < cap && T[(int64_t)order[p] * r + order[p]].x >= thr &&
               T[(int64_t)order[p] * r + order[p]].x >= tfloor) ++p;
        sm.flag = p;
    }
    __syncthreads();
    const int p = sm.flag;
    __syncthreads();
    if (p == 0) return;
    // coefficients g_i = F w_i (K x p) in E, then u_i = X' g_i (NJ x p, FP64) in the output
    for (int64_t idx = t0; idx < (int64_t)K * p; idx += ts) {
        const int i = (int)(idx / p), j = (int)(idx % p);
        double2 acc = make_double2(0.0, 0.0);
        for (int l = 0; l < r; ++l) acc = cadd(acc, cmul(P1[(int64_t)i * r + l], Cm[(int64_t)l * r + order[j]]));
        E[idx] = acc;
    }
    tm.sync();
    double* hdr = in.spawn_out;
    double2* U = (double2*)(hdr + 4 + TTN_SPAWN_MAX_NEW);
    for (int64_t idx = t0; idx < (int64_t)NJ * p; idx += ts) {
        const int J = (int)(idx % NJ), j = (int)(idx / NJ);
        double2 acc = make_double2(0.0, 0.0);
        for (int a = 0; a < A; ++a)
            for (int n = 0; n < chi; ++n)
                acc = cadd(acc, cmul(cd(X[a * smax + (int64_t)J * chi + n]), E[(int64_t)(a * chi + n) * p + j]));
        U[idx] = acc;
    }
    tm.sync();
    // two Gram-Schmidt passes in FP64 against the existing functions and the earlier new ones
    const TS* Ac = (const TS*)op.c;
    for (int j = 0; j < p; ++j) {
        double2* u = U + (int64_t)j * NJ;
        for (int pass = 0; pass < 2; ++pass) {
            for (int n = 0; n < chi + j; ++n) {
                double2 part = make_double2(0.0, 0.0);
                for (int J = t0; J < NJ; J += ts) {
                    const double2 b = n < chi ? cd(Ac[(int64_t)J * chi + n]) : U[(int64_t)(n - chi) * NJ + J];
                    part = cadd(part, cconjmul(b, u[J]));
                }
                const double2 h = team_sum(part, sm, tm);
                for (int J = t0; J < NJ; J += ts) {
                    const double2 b = n < chi ? cd(Ac[(int64_t)J * chi + n]) : U[(int64_t)(n - chi) * NJ + J];
                    u[J] = csub(u[J], cmul(h, b));
                }
                tm.sync();
            }
        }
        double2 part = make_double2(0.0, 0.0);
        for (int J = t0; J < NJ; J += ts) part.x += cabs2(u[J]);
        const double nrm = sqrt(team_sum(part, sm, tm).x);
        for (int J = t0; J < NJ; J += ts) u[J] = cscale(u[J], 1.0 / nrm);
        tm.sync();
    }
    if (threadIdx.x == 0 && tm.rank() == 0) {
        hdr[0] = op.node; hdr[1] = op.child; hdr[2] = p; hdr[3] = NJ;
        for (int j = 0; j < p; ++j) hdr[4 + j] = sqrt(fmax(0.0, T[(int64_t)order[j] * r + order[j]].x));
        __threadfence();
        atomicExch(in.status, TTN_STATUS_SPAWN_HIT);
    }
    tm.sync();
}

// ---------------------------------------------------------------------------
// interpreter: TS = node tensor / bond type, TB = bulk type
// ---------------------------------------------------------------------------
template <class TS, class TB, class TM>
__device__ void run_op(const TtnOp& op, const TtnInstance& in, const TtnOp* opg, const TtnInstance* ing, double dt,
                       Smem& sm, const TM& tm) {
    const int t0 = tm.tid(), ts = tm.nthr();
    const bool lead = threadIdx.x == 0 && tm.rank() == 0;
    Shape sh;
    sh.D = op.D;
    for (int j = 0; j < TTN_MAXD; ++j) sh.d[j] = j < op.D ? op.dims[j] : 1;
    sh.nset = op.nset > 1 ? op.nset : 1;
    TB* work = (TB*)in.work;
    TB* V = work;                                       // TTN_KMAX + 1 Krylov vectors
    TB* t1 = work + (int64_t)(TTN_KMAX + 1) * in.smax;
    TB* t2 = t1 + in.smax;
    TB* t3 = t2 + in.smax;
    double2* Wc = (double2*)(t3 + in.smax);
    double2* Qc = Wc + in.smax;
    const TtnEntry* es = in.entries + op.e0;
    switch (op.type) {
    case TTN_OP_QR_DOWN: {
        TS* A = (TS*)op.a;
        TS* B = (TS*)op.b;
        qr_mode(A, sh, op.k, Wc, Qc, in.qtol, sm, tm);
        const int n = sh.d[op.k];
        const int64_t m = sh.size() / n;
        for (int i = t0; i < n * n; i += ts) {   // B = R^T
            const int a = i / n, b = i % n;
            B[i] = cT<TS>(qr_R(Wc, m, b, a, sm));
        }
        tm.sync();
        break;
    }
    case TTN_OP_QR_UP: {
        TS* A = (TS*)op.a;
        TS* B = (TS*)op.b;
        qr_mode(A, sh, op.k, Wc, Qc, in.qtol, sm, tm);
        const int n = sh.d[op.k];
        const int64_t m = sh.size() / n;
        for (int i = t0; i < n * n; i += ts) {   // B = R
            const int a = i / n, b = i % n;
            B[i] = cT<TS>(qr_R(Wc, m, a, b, sm));
        }
        tm.sync();
        break;
    }
    case TTN_OP_ABSORB_CHILD: {      // A <- A x_last B^T
        TS* A = (TS*)op.a;
        const TS* B = (const TS*)op.b;
        TS* tmp = (TS*)Qc;
        const int n = sh.d[op.k];
        mode_prod(tmp, (const TS*)A, sh.before(op.k), n, n, (int64_t)1, B, true, make_double2(1.0, 0.0), false, tm);
        copy_vec(A, (const TS*)tmp, sh.size(), tm);
        tm.sync();
        break;
    }
    case TTN_OP_ABSORB_PARENT: {     // A <- B x_k A
        TS* A = (TS*)op.a;
        const TS* B = (const TS*)op.b;
        TS* tmp = (TS*)Qc;
        const int n = sh.d[op.k];
        mode_prod(tmp, (const TS*)A, sh.before(op.k), n, n, sh.after(op.k), B, false, make_double2(1.0, 0.0), false, tm);
        copy_vec(A, (const TS*)tmp, sh.size(), tm);
        tm.sync();
        break;
    }
    case TTN_OP_ENV: {                // Krylov vectors are free here: V[0] holds Q, V[1] the chain sum, V[2] P
        const TB* Q = as_bulk<TB>((const TS*)op.a, V, sh.size(), tm);
        const TB* P = op.c ? as_bulk<TB>((const TS*)op.c, V + 2 * in.smax, sh.size(), tm) : Q;
        env_build(Q, P, t1, t2, V + in.smax, sh, op.k, es, op.ne, in.slots, tm);
        break;
    }
    case TTN_OP_COMBO:
        combo<TB>(es, op.ne, in.slots, tm);
        break;
    case TTN_OP_EVOLVE: {
        const int ok = krylov_expm((TS*)op.a, sh, es, op.ne, in.slots, op.tau_coef * dt, op.hermitian, in.ktol,
                                   in.kmax, V, in.smax, t1, t2, t3, sm, tm);
        if (!ok && lead) atomicExch(in.status, 4);   // TTN_E_NOCONV
        tm.sync();
        break;
    }
    case TTN_OP_EIGEN: {
        // residual tolerance: FP64 rounding allows ~1e-12 relative; an FP32 Krylov basis ~1e-7
        const double etol = sizeof(TB) == 16 ? fmax(in.ktol, 1e-12) : fmax(in.ktol, 1e-7);
        double theta = 0.0;
        const int ok = krylov_ground((TS*)op.a, sh, es, op.ne, in.slots, etol, in.kmax, V, in.smax, t1, t2, t3, sm,
                                     &theta, tm);
        if (!ok && lead) atomicExch(in.status, 4);   // TTN_E_NOCONV
        if (ok && lead && op.out) op.out[0] = theta;
        tm.sync();
        break;
    }
    case TTN_OP_DOT: {
        double2 r;
        if (op.ne > 0) {
            const TB* A = as_bulk<TB>((const TS*)op.a, V, sh.vlen(), tm);
            heff_apply(t1, A, t2, V + in.smax, t3, sh, es, op.ne, in.slots, tm);
            r = team_dot(A, (const TB*)t1, sh.vlen(), sm, tm);
        } else {
            const TS* A = (const TS*)op.a;
            r = team_dot(A, A, sh.vlen(), sm, tm);
        }
        if (lead) { op.out[0] = r.x; op.out[1] = r.y; }
        tm.sync();
        break;
    }
    case TTN_OP_CONTRACT_VEC: {      // chain of rectangular mode products, result into slot k
        const TtnEntry e = es[0];
        const TB* cur = as_bulk<TB>((const TS*)op.a, t3, sh.size(), tm);   // t3 is not a chain buffer here
        Shape s2 = sh;
        for (int j = 0; j < sh.D; ++j) {
            if (e.slot[j] < 0) continue;
            const TtnSlot s = in.slots[e.slot[j]];
            TB* dst = (cur == t1) ? t2 : t1;
            mode_prod(dst, cur, s2.before(j), s.cols, s.rows, s2.after(j), (const TB*)s.ptr, false,
                      make_double2(1.0, 0.0), false, tm);
            s2.d[j] = s.rows;
            cur = dst;
        }
        copy_vec((TB*)in.slots[op.k].ptr, cur, s2.size(), tm);
        tm.sync();
        break;
    }
    case TTN_OP_SPAWN:
        spawn_op<TS, TB>(opg, ing, sm, V, in.smax, t1, t2, Wc, Qc, tm);
        break;
    case TTN_OP_PHASE: {             // a <- exp(-i tau_coef dt) a
        TS* A = (TS*)op.a;
        const double th = op.tau_coef * dt;
        const double2 f = make_double2(cos(th), -sin(th));
        for (int64_t i = t0; i < sh.vlen(); i += ts) A[i] = cT<TS>(cmul(f, cd(A[i])));
        tm.sync();
        break;
    }
    case TTN_OP_STEP_END:
        if (lead) {
            const int s = *in.steps_done;
            if (in.stamps) {
                unsigned long long t;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
                in.stamps[s & 4095] = t;
            }
            *in.steps_done = s + 1;
        }
        tm.sync();
        break;
    default:
        if (lead) atomicExch(in.status, 6);
        tm.sync();
        break;
    }
}

__device__ __forceinline__ long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}

template <class TM> __device__ __forceinline__ TM make_team();
template <> __device__ __forceinline__ Solo<256> make_team<Solo<256>>() { return Solo<256>(); }
template <> __device__ __forceinline__ Clu make_team<Clu>() {
    Clu t;
    t.r = (int)cg::this_cluster().block_rank();
    t.n = (int)cg::this_cluster().num_blocks();
    t.par = 0;
    return t;
}

// One team per instance runs its op list nrep times (nrep < 0: the
// instance's own count and time step).  With a slice of device time > 0 a
// team stops after the step that ends its slice; rep_out (optional)
// receives, per instance, the steps run, the status word and the elapsed
// time.  hdr (optional, device memory) supplies the instance count and the
// slice.  Instance b is run by block b (Solo) or by cluster b (Clu).
template <class TS, class TB, class TM>
__global__ void __launch_bounds__(TM::NT, TM::wide ? 1 : 2) program_kernel(const TtnInstance* insts,
                                                                           const TtnLaunchHdr* hdr, int n_inst,
                                                                           double dt, int nrep, long long slice_arg,
                                                                           TtnRepOut* rep_out) {
    __shared__ Smem sm;
    __shared__ long long s_t0;
    const TM tm = make_team<TM>();
    const int b = TM::wide ? (int)(blockIdx.x / tm.size()) : (int)blockIdx.x;
    const int n = hdr ? hdr->n : n_inst;
    const long long slice_ns = hdr ? hdr->slice_ns : slice_arg;
    if (b >= n) return;                       // whole teams leave together
    const TtnInstance in = insts[b];
    const double dtb = nrep < 0 ? in.dt : dt;
    const int nr = nrep < 0 ? in.nrep : nrep;
    if (threadIdx.x == 0) {
        s_flops = 0.0;
        s_flops64 = 0.0;
        s_count = tm.rank() == 0;
        for (int i = 0; i < 8; ++i) s_sub[i] = 0;
        s_t0 = global_ns();
    }
    // (from global memory: indexing the local copy's array would place the
    // whole copy in local memory)
    for (int i = threadIdx.x; i <= TTN_MAXCHI; i += TM::NT) s_mpv[i] = insts[b].mp_variant[i];
#if TTN_WITH_TC
    const bool use_tc = sizeof(TB) == 8 && in.use_tc != 0;
#else
    constexpr bool use_tc = false;           // this build has no tensor-core path
#endif
    if (threadIdx.x == 0) { s_tc_on = use_tc ? 1 : 0; s_tc_phase = 0; s_tc_status = in.status; }
    if (use_tc) {
        if ((threadIdx.x >> 5) == 0) tc_alloc(&s_tc_taddr, kTcCols);
        if (threadIdx.x == 0) {
            tc_mbar_init(&s_tc_bar, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        tc_fence_before();
    }
    tm.sync();
    if (use_tc) tc_fence_after();
    int rep = 0;
    bool stopped = false;
    while (rep < nr) {
        for (int o = 0; o < in.n_ops; ++o) {
            const int st = team_flag(threadIdx.x == 0 ? *((volatile int*)in.status) : 0, sm, tm);
            if (st != 0) { stopped = true; break; }
            const TtnOp op = in.ops[o];
            const long long c0 = clock64();
            run_op<TS, TB>(op, in, in.ops + o, insts + b, dtb, sm, tm);
            if (threadIdx.x == 0 && s_count && in.op_cycles)
                atomicAdd(&in.op_cycles[op.type & 15], (unsigned long long)(clock64() - c0));
        }
        if (stopped) break;
        ++rep;
        if (slice_ns > 0) {
            const int stop = team_flag(threadIdx.x == 0 ? (int)(global_ns() - s_t0 >= slice_ns) : 0, sm, tm);
            if (stop) break;
        }
    }
    if (threadIdx.x == 0 && s_count && in.flops) {
        atomicAdd(in.flops, s_flops);
        atomicAdd(in.flops + 1, s_flops64);
    }
    if (threadIdx.x == 0 && s_count && in.op_cycles)
        for (int i = 0; i < 8; ++i) atomicAdd(&in.op_cycles[16 + i], s_sub[i]);
    if (threadIdx.x == 0 && s_count && rep_out) {
        TtnRepOut r;
        r.reps = rep;
        r.status = *((volatile int*)in.status);
        r.elapsed_ns = global_ns() - s_t0;
        rep_out[b] = r;
    }
    if (use_tc) {                             // every MMA was waited for: free the tensor memory
        tc_fence_before();
        __syncthreads();
        if ((threadIdx.x >> 5) == 0) tc_dealloc(s_tc_taddr, kTcCols);
    }
    if constexpr (TM::wide) tm.sync();        // no block leaves while others may read its shared memory
}

}  // namespace
