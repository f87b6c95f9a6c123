// Device helpers shared by the single-system and the batched Bi-CGSTAB
// solvers: the tile mapping of the stencil kernels, the shared-memory
// stencil application (FP64 matrix form, compensated FP32 difference form),
// deterministic block reductions (FP64 and double-float), and the grid
// barrier state of the persistent launches.
#pragma once

#include "common.cuh"

namespace mcd {

// Grid barrier state: per block an arrival flag, and a release word on a
// 128-byte line of its own (polling one shared word from every block queues
// the polls on one L2 slice and delays the wake-up of the last blocks by
// microseconds).  Both hold barrier epochs 1, 2, ... within a launch (the
// host zeroes them before each launch), so nothing is reset in between.
struct GridBarrier {
    unsigned int pad[64];
    unsigned int flag[1];     // [grid] arrival epochs, then the release lines
};

__host__ __device__ __forceinline__ size_t barrier_release_offset(int grid) {
    return ((size_t)grid * sizeof(unsigned int) + 127) / 128 * 128;
}

// Bytes of a barrier for `grid` blocks.
__host__ __device__ __forceinline__ size_t barrier_bytes(int grid) {
    return sizeof(GridBarrier) + barrier_release_offset(grid) + (size_t)grid * 128;
}

__device__ __forceinline__ unsigned *release_word(GridBarrier *bar, int grid, int block) {
    return (unsigned *)((char *)bar->flag + barrier_release_offset(grid)) + (size_t)block * 32;
}

template <typename F>
__device__ __forceinline__ F vload(const F *p) {
    return *((volatile const F *)p);
}

// Tile of the Bi-CGSTAB stencil kernels: 256 threads own X x Y (x Z) DPs, R
// per thread, strided along the last tiled axis (thread grid X x TY x TZ).
// Grid-barrier flag accesses at GPU scope: a release store publishes every
// write that precedes it (the block's writes, ordered by the __syncthreads in
// front of it), an acquire load makes them visible to the polling thread,
// and the __syncthreads after the poll hands them to the rest of its block.
__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_relaxed_u32(unsigned *p, unsigned v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait until *p == v: back-to-back polls first, then polls spaced by
// __nanosleep.  Returns false after `limit` polls.
__device__ __forceinline__ bool wait_eq(const unsigned *p, unsigned v, long long limit) {
    long long polls = 0;
    while (ld_acquire(p) != v) {
        if (++polls > limit) return false;
        if (polls > 256) __nanosleep(64);
    }
    return true;
}

// Tile of DPs one block works on (X x Y x Z cells; each thread owns R rows,
// TY / TZ apart), for the stencil shape G of common.cuh.
template <int G> struct Tile;
template <> struct Tile<2> {
    static constexpr int X = 32, Y = 16, Z = 1, R = 2, TY = 8, TZ = 1;
};
template <> struct Tile<3> {
    static constexpr int X = 32, Y = 4, Z = 4, R = 2, TY = 4, TZ = 2;
};
// 9x9: 64 x 8 tiles, so that each row of a tile's weights is a 256-byte
// segment of the slot-major rows (the rows come from HBM).
template <> struct Tile<9> {
    static constexpr int X = 64, Y = 8, Z = 1, R = 2, TY = 4, TZ = 1;
};

// The tile plus its halo of Shape<G>::R cells on every side.
template <int G> struct HaloDims {
    static constexpr int RH = Shape<G>::R;
    static constexpr int HX = Tile<G>::X + 2 * RH;
    static constexpr int HY = Tile<G>::Y + 2 * RH;
    static constexpr int HZ = (Shape<G>::dim == 3) ? Tile<G>::Z + 2 * RH : 1;
    static constexpr int H = HX * HY * HZ;
    static constexpr int S = Shape<G>::S;
};

__device__ __forceinline__ int wrap_clamp(int v, int n, int per) {
    if (v < 0) return per ? v + n : 0;
    if (v >= n) return per ? v - n : n - 1;
    return v;
}

// Deterministic block reduction of NV values; thread 0 writes them to
// partials[q * stride + block].
template <int NV, typename A>
__device__ __forceinline__ void block_partials(A (&v)[NV], double *partials, int stride, int block) {
    __shared__ double wsum[NV][32];
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
#pragma unroll
    for (int q = 0; q < NV; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    if ((tid & 31) == 0)
        for (int q = 0; q < NV; ++q) wsum[q][tid >> 5] = (double)v[q];
    __syncthreads();
    if (tid < 32) {
        const int nw = nthreads >> 5;
        for (int q = 0; q < NV; ++q) {
            double x = (tid < nw) ? wsum[q][tid] : 0.0;
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (tid == 0) partials[q * stride + block] = x;
        }
    }
}

// ---- compensated FP32 dot products --------------------------------------
// FP32 kernels accumulate each dot product as an unevaluated pair (hi, lo):
// products are split exactly with fma and added with TwoSum, warps and the
// block combine pairs the same way, and one thread per block converts the
// pair to FP64.  The sums are then accurate to about twice FP32 precision
// relative to sum |a_i b_i|, so rho = r^.r stays meaningful when it is much
// smaller than |r^||r| (as the residual migrates away from r^), and no
// per-thread FP64 work (slow on this GPU) is needed.
struct DF {
    float hi, lo;
};

// The error-free steps use the _rn intrinsics, which the compiler never
// contracts into fused multiply-adds (contraction would change the rounded
// product that TwoSum has to see and void the error terms).
__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void df_add_prod(DF &acc, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -p);
    float e;
    two_sum_f(acc.hi, p, acc.hi, e);
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, pe));
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
    DF r;
    float e;
    two_sum_f(a.hi, b.hi, r.hi, e);
    r.lo = __fadd_rn(__fadd_rn(e, a.lo), b.lo);
    return r;
}

__device__ __forceinline__ DF df_shfl_down(DF x, int o) {
    return DF{__shfl_down_sync(0xffffffffu, x.hi, o), __shfl_down_sync(0xffffffffu, x.lo, o)};
}

template <int NV>
__device__ __forceinline__ void block_partials_df(DF (&v)[NV], double *partials, int stride, int block) {
    __shared__ DF wsum[NV][32];
    const int tid = threadIdx.x;
    const int nthreads = blockDim.x;
#pragma unroll
    for (int q = 0; q < NV; ++q)
        for (int o = 16; o > 0; o >>= 1) {
            DF other;
            other.hi = __shfl_down_sync(0xffffffffu, v[q].hi, o);
            other.lo = __shfl_down_sync(0xffffffffu, v[q].lo, o);
            v[q] = df_add(v[q], other);
        }
    if ((tid & 31) == 0)
        for (int q = 0; q < NV; ++q) wsum[q][tid >> 5] = v[q];
    __syncthreads();
    if (tid < 32) {
        const int nw = nthreads >> 5;
        for (int q = 0; q < NV; ++q) {
            DF x = (tid < nw) ? wsum[q][tid] : DF{0.0f, 0.0f};
            for (int o = 16; o > 0; o >>= 1) {
                DF other;
                other.hi = __shfl_down_sync(0xffffffffu, x.hi, o);
                other.lo = __shfl_down_sync(0xffffffffu, x.lo, o);
                x = df_add(x, other);
            }
            if (tid == 0) partials[q * stride + block] = (double)x.hi + (double)x.lo;
        }
    }
}

// Accumulator of one dot product: FP64 for the FP64 kernels, a compensated
// pair for the FP32 ones.
template <typename T> struct DotAcc;
template <> struct DotAcc<double> {
    double v = 0.0;
    __device__ void add(double a, double b) { v += a * b; }
};
template <> struct DotAcc<float> {
    DF v{0.0f, 0.0f};
    __device__ void add(float a, float b) { df_add_prod(v, a, b); }
};

template <int NV>
__device__ __forceinline__ void dot_partials(DotAcc<double> (&d)[NV], double *partials, int stride, int block) {
    double v[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = d[q].v;
    block_partials<NV, double>(v, partials, stride, block);
}

template <int NV>
__device__ __forceinline__ void dot_partials(DotAcc<float> (&d)[NV], double *partials, int stride, int block) {
    DF v[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = d[q].v;
    block_partials_df<NV>(v, partials, stride, block);
}

// Returns true in the block that arrives last; that block then holds the
// totals of the NV partial sums in out[] (valid in every thread).  The
// partials are read with independent loads, four per thread per round, so
// the tail costs about one L2 round trip for the few-hundred-block grids the
// solver launches.
template <int NV>
__device__ __forceinline__ bool last_block_totals(const double *partials, int stride, int nblocks,
                                                  unsigned int *counter, double (&out)[NV]) {
    __shared__ bool is_last;
    __shared__ double red[NV][32];
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    if (tid == 0) {
        __threadfence();
        const unsigned t = atomicAdd(counter, 1u);
        is_last = (t == (unsigned)nblocks - 1u);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = 0.0;
    for (int b0 = tid; b0 < nblocks; b0 += 4 * nthreads) {
        double v[NV][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int b = b0 + u * nthreads;
#pragma unroll
            for (int q = 0; q < NV; ++q) v[q][u] = (b < nblocks) ? __ldcg(partials + q * stride + b) : 0.0;
        }
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] += (v[q][0] + v[q][1]) + (v[q][2] + v[q][3]);
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_down_sync(0xffffffffu, acc[q], o);
        if ((tid & 31) == 0) red[q][tid >> 5] = acc[q];
    }
    __syncthreads();
    for (int q = 0; q < NV; ++q) {
        double x = 0.0;
        for (int w = 0; w < (nthreads >> 5); ++w) x += red[q][w];
        out[q] = x;
    }
    if (tid == 0) *counter = 0u;
    return true;
}

struct TileArgs {
    Geo g;
    int bx, by, bz;      // tiles per axis
    int ntiles;
    const int8_t *kind;  // non-NULL: Neumann rows act as identity rows
};

template <int G>
__device__ __forceinline__ void tile_origin(const TileArgs &ta, int tile, int &x0, int &y0, int &z0) {
    const int tx = tile % ta.bx;
    const int rest = tile / ta.bx;
    const int ty = rest % ta.by;
    const int tz = rest / ta.by;
    x0 = tx * Tile<G>::X;
    y0 = ty * Tile<G>::Y;
    z0 = tz * Tile<G>::Z;
}

// Global index of halo element h of the tile at (x0, y0, z0).
template <int G>
__device__ __forceinline__ int64_t halo_index(const Geo &g, int h, int x0, int y0, int z0) {
    using HD = HaloDims<G>;
    const int hx = h % HD::HX;
    const int hy = (h / HD::HX) % HD::HY;
    const int hz = h / (HD::HX * HD::HY);
    const int gx = wrap_clamp(x0 + hx - HD::RH, g.n[0], g.per[0]);
    const int gy = wrap_clamp(y0 + hy - HD::RH, g.n[1], g.per[1]);
    if (Shape<G>::dim == 2) return (int64_t)gx + (int64_t)g.n[0] * gy;
    const int gz = wrap_clamp(z0 + hz - HD::RH, g.n[2], g.per[2]);
    return (int64_t)gx + (int64_t)g.n[0] * ((int64_t)gy + (int64_t)g.n[1] * gz);
}

// DP r of thread tid in the tile at (x0, y0, z0): global index, or -1
// outside the mesh; (lx, ly, lz) are its coordinates inside the tile.
template <int G>
__device__ __forceinline__ int64_t tile_dp(const Geo &g, int tid, int r, int x0, int y0, int z0, int &lx,
                                           int &ly, int &lz) {
    using TL = Tile<G>;
    constexpr int DIM = Shape<G>::dim;
    lx = tid % TL::X;
    if (DIM == 2) {
        ly = (tid / TL::X) + r * TL::TY;
        lz = 0;
    } else {
        ly = (tid / TL::X) % TL::TY;
        lz = tid / (TL::X * TL::TY) + r * TL::TZ;
    }
    const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
    if (gx >= g.n[0] || gy >= g.n[1] || (DIM == 3 && gz >= g.n[2])) return -1;
    return (DIM == 2) ? (int64_t)gx + (int64_t)g.n[0] * gy
                      : (int64_t)gx + (int64_t)g.n[0] * ((int64_t)gy + (int64_t)g.n[1] * gz);
}

template <int G>
__device__ __forceinline__ int tile_centre(int lx, int ly, int lz) {
    using HD = HaloDims<G>;
    return (lx + HD::RH) + HD::HX * ((ly + HD::RH) + HD::HY * (lz + (Shape<G>::dim == 3 ? HD::RH : 0)));
}

// (A x)_k from the shared-memory tile of x and the row weights w[] (already
// in registers).  FP64 rows are in matrix form (sum_s c_s x_s); FP32 rows in
// difference form (c_C x_k + sum_{s != C} c_s (x_s - x_k), centre slot = row
// sum), which keeps the O(1/l0^2) weights from cancelling away the FP32
// mantissa.
//
// The FP32 form is also compensated: each product c_s (x_s - x_k) is split
// exactly into p + e with a fused multiply-add, and the products are summed
// with Knuth's TwoSum into a (hi, lo) pair, so the row is accumulated to
// about twice FP32 precision and rounded once.  A plain FP32 sum of the
// O(|grad x| / l0) terms loses the digits of their O(lap x) sum and slows
// Bi-CGSTAB by about 2x; the compensation costs about 11 FP32 operations per
// term, which this bandwidth-bound kernel has to spare.
//
// COMP = false accumulates the FP32 difference form with one FMA per term
// instead.  The single-system 2D solver uses it: its iteration is bound by
// issue and latency, not bandwidth, and with its dot products still
// double-float the plain 3x3 sum costs about 4 % more iterations on the
// flow's PPE while each iteration takes about 9 % less.  Wide and 3D
// stencils and the batched solver keep the compensated sum.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

template <int G, typename T, bool COMP = true>
__device__ __forceinline__ T stencil_apply(const T *w, const T *tile, int lx, int ly, int lz) {
    using HD = HaloDims<G>;
    constexpr int C = HD::S / 2, W = Shape<G>::W;
    const T xk = tile[tile_centre<G>(lx, ly, lz)];
    if (sizeof(T) == 4 && !COMP) {
        float acc = (float)w[C] * (float)xk;   // centre weight is 0 or 1: exact
#pragma unroll
        for (int s = 0; s < HD::S; ++s) {
            if (s == C) continue;
            const int ox = s % W, oy = (s / W) % W, oz = s / (W * W);
            const int h = (lx + ox) + HD::HX * ((ly + oy) + HD::HY * (lz + oz));
            acc = __fmaf_rn((float)w[s], __fsub_rn((float)tile[h], (float)xk), acc);
        }
        return (T)acc;
    }
    if (sizeof(T) == 4) {
        float hi = (float)w[C] * (float)xk, lo = 0.0f;   // centre weight is 0 or 1: exact
#pragma unroll
        for (int s = 0; s < HD::S; ++s) {
            if (s == C) continue;
            const int ox = s % W, oy = (s / W) % W, oz = s / (W * W);
            const int h = (lx + ox) + HD::HX * ((ly + oy) + HD::HY * (lz + oz));
            const float d = __fsub_rn((float)tile[h], (float)xk);
            const float p = __fmul_rn((float)w[s], d);
            const float pe = __fmaf_rn((float)w[s], d, -p);
            float e;
            two_sum(hi, p, hi, e);
            lo = __fadd_rn(lo, __fadd_rn(e, pe));
        }
        return (T)__fadd_rn(hi, lo);
    }
    T acc = (T)0;
#pragma unroll
    for (int s = 0; s < HD::S; ++s) {
        const int ox = s % W, oy = (s / W) % W, oz = s / (W * W);
        const int h = (lx + ox) + HD::HX * ((ly + oy) + HD::HY * (lz + oz));
        acc += w[s] * tile[h];
    }
    return acc;
}

// stencil_apply for wide stencils (81 weights per row): each weight is read
// from the slot-major rows where it is used, instead of staging the whole
// row in registers.  The FP32 difference form keeps the compensated
// (double-float) sum, but over NA independent (hi, lo) accumulators (slot s
// goes to accumulator s % NA), merged with TwoSum at the end: one chain of 80
// dependent TwoSums left the SM waiting on latency.
template <int G, typename T>
__device__ __forceinline__ T stencil_apply_rows(const T *__restrict__ row, int64_t N, int64_t k, const T *tile,
                                                int lx, int ly, int lz) {
    using HD = HaloDims<G>;
    constexpr int C = HD::S / 2, W = Shape<G>::W;
    const T xk = tile[tile_centre<G>(lx, ly, lz)];
    const T *rk = row + k;
    if (sizeof(T) == 4) {
        constexpr int NA = 4;
        float hi[NA], lo[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) { hi[a] = 0.0f; lo[a] = 0.0f; }
        hi[C % NA] = (float)__ldg(rk + (int64_t)C * N) * (float)xk;   // centre weight is 0 or 1: exact
#pragma unroll
        for (int s = 0; s < HD::S; ++s) {
            if (s == C) continue;
            const int ox = s % W, oy = (s / W) % W, oz = s / (W * W);
            const int h = (lx + ox) + HD::HX * ((ly + oy) + HD::HY * (lz + oz));
            const float ws = (float)__ldg(rk + (int64_t)s * N);
            const float d = __fsub_rn((float)tile[h], (float)xk);
            const float p = __fmul_rn(ws, d);
            const float pe = __fmaf_rn(ws, d, -p);
            float e;
            two_sum(hi[s % NA], p, hi[s % NA], e);
            lo[s % NA] = __fadd_rn(lo[s % NA], __fadd_rn(e, pe));
        }
        float h01, e01, h23, e23, hs, es;
        two_sum(hi[0], hi[1], h01, e01);
        two_sum(hi[2], hi[3], h23, e23);
        two_sum(h01, h23, hs, es);
        const float lsum = __fadd_rn(__fadd_rn(__fadd_rn(lo[0], lo[1]), __fadd_rn(lo[2], lo[3])),
                                     __fadd_rn(__fadd_rn(e01, e23), es));
        return (T)__fadd_rn(hs, lsum);
    }
    T acc[3] = {(T)0, (T)0, (T)0};
#pragma unroll
    for (int s = 0; s < HD::S; ++s) {
        const int ox = s % W, oy = (s / W) % W, oz = s / (W * W);
        const int h = (lx + ox) + HD::HX * ((ly + oy) + HD::HY * (lz + oz));
        acc[s % 3] += __ldg(rk + (int64_t)s * N) * tile[h];
    }
    return (acc[0] + acc[1]) + acc[2];
}

// Row weights of DP k into registers (zeros for k < 0).
template <int S, typename T>
__device__ __forceinline__ void load_row(const T *__restrict__ row, int64_t N, int64_t k, T *w) {
#pragma unroll
    for (int s = 0; s < S; ++s) w[s] = (k >= 0) ? __ldg(row + (int64_t)s * N + k) : (T)0;
}

}  // namespace mcd
