// cnn.cu - the learned warm start of the pressure solve (not in the paper):
// a stack of 3x3 convolutions on the background-mesh grid, run on the bf16
// tensor cores with FP32 accumulation, its training step (backward pass,
// Adam) and the warm start p <- p + s e, e = network correction, s the
// residual-minimising step along e.
//
// Data layout (HBM): activations channels-last bf16 [N][C] with C = 8 for the
// input features and the output gradient, 32 for hidden layers; the FP32
// master parameters, gradients and Adam moments use the flat layout of the
// C ABI (per layer W[o][c][dj][di], then b[o]).  Each layer keeps a packed
// bf16 copy of its weights in the shared-memory layout of the convolution
// kernel ([out channel][tap * C_in + c], padded), plus the tap-flipped,
// transposed copy that turns the input-gradient pass into the same kernel.
//
// Convolution as an implicit GEMM: a CTA computes a 16 x 16 cell tile for all
// output channels.  The input tile with its one-cell halo and the packed
// weights are staged in shared memory; warp w owns tile rows 2w and 2w+1 (two
// m16 row blocks), K runs over (tap, input channel) in steps of 16, and every
// step issues mma.m16n8k16 (bf16 x bf16 -> f32).  Row strides are padded so
// that the 32-bit fragment loads of a warp touch 32 distinct banks.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace mcd {
namespace cnn {

typedef __nv_bfloat16 bf16;

constexpr int TW = 16, TH = 16, HW = TW + 2, HH = TH + 2, NTHR = 256;
constexpr int FEAT = 8;         // stored input channels (7 features + 1 zero)
constexpr int WIDTH = 32;
constexpr int MAX_LAYERS = 8;
constexpr int RED_BLOCKS = 608;   // grid of the reduction kernels: 4 CTAs x 152 SMs
constexpr int RED_THREADS = 256;
constexpr int NRED = 6;           // values reduced per block

__host__ __device__ constexpr int kpad(int cinp) { return (9 * cinp + 15) / 16 * 16; }
// Row stride (bf16) of a [rows][K] operand: kpad/2 words is a multiple of 8,
// so +4 words puts the 8 rows of a fragment load 4*odd words apart.
__host__ __device__ constexpr int kstr(int cinp) { return kpad(cinp) + 8; }
// Per-cell channel stride of the staged input tile (same bank argument).
__host__ __device__ constexpr int cstr(int cinp) { return cinp == 8 ? 8 : cinp + 8; }
__host__ __device__ constexpr size_t conv_smem(int cinp, int coutp) {
    return (size_t)coutp * kstr(cinp) * 2 + (size_t)HH * HW * cstr(cinp) * 2;
}
constexpr int WG_GS = TW * TH + 8;   // row stride of the transposed gradient tile
constexpr int WG_XP = HH * TW + 8;   // plane stride of the shifted input copies
__host__ __device__ constexpr int wg_rows(int coutp) { return coutp >= 16 ? coutp : 16; }
__host__ __device__ constexpr size_t wgrad_smem(int cinp, int coutp) {
    return (size_t)wg_rows(coutp) * WG_GS * 2 + (size_t)3 * cinp * WG_XP * 2 + 8 * 32 * 4;
}
__host__ __device__ constexpr int64_t wg_part_stride(int cinp, int coutp) {
    return (int64_t)9 * coutp * cinp + coutp;
}

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ uint32_t lds32(const bf16 *p) {
    return *reinterpret_cast<const uint32_t *>(p);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------------------
// Convolution (forward layer, or input-gradient pass with flipped weights)
// ---------------------------------------------------------------------------
enum { EPI_RELU = 0, EPI_LAST = 1, EPI_DGRAD = 2 };

struct ConvArgs {
    const bf16 *in;      // [N][CINP]
    const bf16 *w;       // [COUTP][kstr(CINP)] packed
    const float *bias;   // [COUTP] (EPI_RELU, EPI_LAST)
    const bf16 *gate;    // [N][COUTP] (EPI_DGRAD): forward activation, passes where > 0
    bf16 *out;           // [N][COUTP] (EPI_RELU, EPI_DGRAD)
    float *out32;        // [N] channel 0 (EPI_LAST)
    int nx, ny;
};

template <int CINP, int COUTP, int EPI>
__global__ void __launch_bounds__(NTHR) conv_kernel(ConvArgs a) {
    constexpr int KP = kpad(CINP), KS = kstr(CINP), CS = cstr(CINP);
    constexpr int NT = COUTP / 8, QCH = CINP / 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    bf16 *wsm = reinterpret_cast<bf16 *>(smem_raw);
    bf16 *hsm = wsm + COUTP * KS;
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.w);
        uint4 *dst = reinterpret_cast<uint4 *>(wsm);
        for (int i = tid; i < COUTP * KS / 8; i += NTHR) dst[i] = src[i];
    }
    for (int i = tid; i < HH * HW * QCH; i += NTHR) {
        const int cell = i / QCH, q = i - cell * QCH;
        const int hr = cell / HW, hc = cell - hr * HW;
        const int gy = y0 + hr - 1, gx = x0 + hc - 1;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (gy >= 0 && gy < a.ny && gx >= 0 && gx < a.nx)
            v = reinterpret_cast<const uint4 *>(a.in)[((int64_t)gy * a.nx + gx) * QCH + q];
        *reinterpret_cast<uint4 *>(hsm + cell * CS + q * 8) = v;
    }
    __syncthreads();

    const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    float acc[2][NT][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[mt][nt][q] = 0.0f;

#pragma unroll
    for (int ks = 0; ks < KP / 16; ++ks) {
        const int kL = ks * 16, kH = kL + 8;
        const int tapL = kL / CINP, cL = kL % CINP, tapH = kH / CINP, cH = kH % CINP;
        uint32_t b[NT][2];
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const bf16 *wr = wsm + (nt * 8 + g) * KS + 2 * t;
            b[nt][0] = lds32(wr + kL);
            b[nt][1] = lds32(wr + kH);
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int r = warp * 2 + mt;
            uint32_t a0 = 0u, a1 = 0u, a2 = 0u, a3 = 0u;
            if (tapL < 9) {
                const bf16 *hp = hsm + ((r + tapL / 3) * HW + g + tapL % 3) * CS + cL + 2 * t;
                a0 = lds32(hp);
                a1 = lds32(hp + 8 * CS);
            }
            if (tapH < 9) {
                const bf16 *hp = hsm + ((r + tapH / 3) * HW + g + tapH % 3) * CS + cH + 2 * t;
                a2 = lds32(hp);
                a3 = lds32(hp + 8 * CS);
            }
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) mma_bf16(acc[mt][nt], a0, a1, a2, a3, b[nt][0], b[nt][1]);
        }
    }

#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        const int gy = y0 + warp * 2 + mt;
        if (gy >= a.ny) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int gx = x0 + g + 8 * h;
            if (gx >= a.nx) continue;
            const int64_t cell = (int64_t)gy * a.nx + gx;
            if constexpr (EPI == EPI_LAST) {
                if (t == 0) a.out32[cell] = acc[mt][0][2 * h] + a.bias[0];
            } else {
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const int ch = nt * 8 + 2 * t;
                float v0 = acc[mt][nt][2 * h], v1 = acc[mt][nt][2 * h + 1];
                if (EPI == EPI_RELU) {
                    v0 = fmaxf(v0 + a.bias[ch], 0.0f);
                    v1 = fmaxf(v1 + a.bias[ch + 1], 0.0f);
                } else {
                    const __nv_bfloat162 gt =
                        *reinterpret_cast<const __nv_bfloat162 *>(a.gate + cell * COUTP + ch);
                    if (!(__low2float(gt) > 0.0f)) v0 = 0.0f;
                    if (!(__high2float(gt) > 0.0f)) v1 = 0.0f;
                }
                *reinterpret_cast<__nv_bfloat162 *>(a.out + cell * COUTP + ch) =
                    __floats2bfloat162_rn(v0, v1);
            }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Hidden 32 -> 32 convolution on the 5th-generation tensor cores
// (tcgen05.mma, bf16 operands from shared memory, FP32 accumulators in
// tensor memory).  One CTA (one warpgroup) computes a 16 x 16 cell tile as
// two M = 128 (16 rows x 8 columns) by N = 32 accumulators.  The input tile
// and its halo are staged as 8-cell x 16-byte core matrices
// ([row][channel chunk][column][8 channels]), so the A operand of tap
// (dj, di) is the same layout started dj rows and di cells further: every
// MMA is a descriptor with a shifted start address.  The weights are read
// from the packed [out][tap * 32 + c] copy, whose 8-channel runs are the
// 16-byte rows of the B core matrices.  K = 9 taps x 32 channels in 18 MMAs
// of K = 16 per accumulator.  The completion of the MMAs is signalled by
// tcgen05.commit on an mbarrier whose wait is bounded; a wait that gives up
// sets *err and skips the epilogue (the tensor memory is freed either way).
// ---------------------------------------------------------------------------
namespace tc {
constexpr int HX = TW + 2, HY = TH + 2;         // 18 x 18 halo
constexpr int RS = 4 * HX * 16;                  // bytes per halo row (4 chunks x 18 cells)
constexpr int CQ = HX * 16;                      // bytes per chunk plane of a row
constexpr int HALO = HY * RS;                    // 20736
constexpr int WB = 9 * 4 * 32 * 16;              // 18432: [tap][chunk][out][8]
constexpr size_t SMEM = (size_t)WB + 2 * HALO;
constexpr int NCOL = 64;                         // two accumulators of 32 columns
}  // namespace tc

// Shared-memory matrix descriptor: start address, leading byte offset (the
// stride between core matrices along K), stride byte offset (between core
// matrices along M or N), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Epilogue of one accumulator stage: warp w reads tensor-memory lanes
// 32 (w % 4) .. + 31 of accumulator h = w / 4 (tile columns 8 h .. 8 h + 7);
// lane row m is tile cell (m / 8, 8 h + m % 8).
template <int EPI>
__device__ __forceinline__ void tc_epilogue(const ConvArgs &a, uint32_t tacc, int x0, int y0) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int h = warp >> 2, quad = warp & 3;
    uint32_t r[32];
    const uint32_t taddr = tacc + ((uint32_t)(quad * 32) << 16) + h * 32;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int m = quad * 32 + lane;
    const int gy = y0 + (m >> 3), gx = x0 + 8 * h + (m & 7);
    if (gy >= a.ny || gx >= a.nx) return;
    const int64_t cell = (int64_t)gy * a.nx + gx;
    float v[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
    if constexpr (EPI == EPI_RELU) {
#pragma unroll
        for (int c = 0; c < 32; ++c) v[c] = fmaxf(v[c] + a.bias[c], 0.0f);
    } else {
        const uint4 *gp = reinterpret_cast<const uint4 *>(a.gate + cell * 32);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint4 gv = gp[j];
            const bf16 *ge = reinterpret_cast<const bf16 *>(&gv);
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (!(__bfloat162float(ge[e]) > 0.0f)) v[8 * j + e] = 0.0f;
        }
    }
    uint4 *op = reinterpret_cast<uint4 *>(a.out + cell * 32);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint4 o;
        o.x = pack2(__float2bfloat16_rn(v[8 * j + 0]), __float2bfloat16_rn(v[8 * j + 1]));
        o.y = pack2(__float2bfloat16_rn(v[8 * j + 2]), __float2bfloat16_rn(v[8 * j + 3]));
        o.z = pack2(__float2bfloat16_rn(v[8 * j + 4]), __float2bfloat16_rn(v[8 * j + 5]));
        o.w = pack2(__float2bfloat16_rn(v[8 * j + 6]), __float2bfloat16_rn(v[8 * j + 7]));
        op[j] = o;
    }
}

// Bounded wait for phase `parity` of an mbarrier; false if it gave up.
__device__ __forceinline__ bool tc_wait(uint32_t mbar_a, uint32_t parity) {
    for (long long polls = 0; polls < (1ll << 22); ++polls) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar_a), "r"(parity));
        if (done) return true;
    }
    return false;
}

// Copy the input tile of (x0, y0) with its halo into `halo` in the
// core-matrix layout, 16-byte asynchronous copies; chunks outside the grid
// read 0 bytes and are zero-filled.
__device__ __forceinline__ void tc_stage(const ConvArgs &a, unsigned char *halo, int x0, int y0) {
    for (int i = threadIdx.x; i < tc::HY * tc::HX * 4; i += 256) {
        const int cell = i >> 2, q = i & 3, hy = cell / tc::HX, hx = cell - hy * tc::HX;
        const int gy = y0 + hy - 1, gx = x0 + hx - 1;
        const bool in = gy >= 0 && gy < a.ny && gx >= 0 && gx < a.nx;
        const uint4 *src = reinterpret_cast<const uint4 *>(a.in) + (in ? ((int64_t)gy * a.nx + gx) * 4 + q : 0);
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(halo + (hy * 4 + q) * tc::CQ + hx * 16);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(in ? 16 : 0)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Persistent CTAs (256 threads): the weights are staged once; tiles are
// taken in a grid-stride loop with two halo buffers and two accumulator
// stages.  While the MMAs of tile i run on the tensor core, the halo of
// tile i + 1 is copied asynchronously and the epilogue of tile i - 1 runs.
template <int EPI>
__global__ void __launch_bounds__(256) conv_tc_kernel(ConvArgs a, int *err) {
    static_assert(EPI == EPI_RELU || EPI == EPI_DGRAD, "hidden-layer epilogues only");
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char *wsm = tc_smem;
    unsigned char *hbuf = tc_smem + tc::WB;        // two halo buffers
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int tiles_x = (a.nx + TW - 1) / TW;
    const int ntiles = tiles_x * ((a.ny + TH - 1) / TH);
    constexpr int KS = kstr(WIDTH);   // row stride (bf16) of the packed weights
    for (int i = tid; i < 9 * 4 * 32; i += 256) {
        const int t = i >> 7, rem = i & 127, q = rem >> 5, n = rem & 31;
        *reinterpret_cast<uint4 *>(wsm + ((t * 4 + q) * 32 + n) * 16) =
            *reinterpret_cast<const uint4 *>(a.w + (size_t)n * KS + t * WIDTH + q * 8);
    }
    const uint32_t mb0 = (uint32_t)__cvta_generic_to_shared(&mbar[0]);
    const uint32_t mb1 = (uint32_t)__cvta_generic_to_shared(&mbar[1]);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb1));
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&tmem_base)),
                     "n"(2 * tc::NCOL));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    const uint32_t wbase = (uint32_t)__cvta_generic_to_shared(wsm);
    const uint32_t hbase0 = (uint32_t)__cvta_generic_to_shared(hbuf);
    // D f32, A and B bf16, both K-major, N = 32, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
    uint32_t phase0 = 0, phase1 = 0;
    int prev_tile = -1, prev_s = 0;
    bool ok = true;
    if (blockIdx.x < ntiles)
        tc_stage(a, hbuf, (blockIdx.x % tiles_x) * TW, (blockIdx.x / tiles_x) * TH);
    for (int it = 0, tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++it) {
        const int s = it & 1;
        // the MMAs of tile i - 1 are done before its halo buffer is refilled
        bool prev_done = true;
        if (prev_tile >= 0) {
            prev_done = tc_wait(prev_s ? mb1 : mb0, prev_s ? phase1 : phase0);
            if (prev_s) phase1 ^= 1u; else phase0 ^= 1u;
        }
        ok = __syncthreads_and(prev_done);
        if (!ok) break;
        const int next = tile + gridDim.x;
        if (next < ntiles) tc_stage(a, hbuf + (s ^ 1) * tc::HALO, (next % tiles_x) * TW, (next / tiles_x) * TH);
        else asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");   // this tile's halo has landed
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // staged tile -> tensor core
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t tmem = tmem_base;
        if (tid == 0) {
            const uint32_t hb = hbase0 + s * tc::HALO;
            for (int h = 0; h < 2; ++h)
                for (int t = 0; t < 9; ++t)
                    for (int k2 = 0; k2 < 2; ++k2) {
                        const uint32_t aaddr = hb + (t / 3) * tc::RS + 2 * k2 * tc::CQ + (8 * h + t % 3) * 16;
                        const uint32_t baddr = wbase + (t * 4 + 2 * k2) * 512;
                        const uint64_t ad = tc_desc(aaddr, tc::CQ, tc::RS), bd = tc_desc(baddr, 512, 128);
                        const uint32_t accum = (t | k2) ? 1u : 0u;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(
                                tmem + s * tc::NCOL + h * 32),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                    }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                s ? mb1 : mb0));
        }
        if (prev_tile >= 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            tc_epilogue<EPI>(a, tmem + prev_s * tc::NCOL, (prev_tile % tiles_x) * TW, (prev_tile / tiles_x) * TH);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        }
        prev_tile = tile;
        prev_s = s;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (ok && prev_tile >= 0) {
        const bool done = tc_wait(prev_s ? mb1 : mb0, prev_s ? phase1 : phase0);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        ok = __syncthreads_and(done);
        if (ok)
            tc_epilogue<EPI>(a, tmem_base + prev_s * tc::NCOL, (prev_tile % tiles_x) * TW,
                             (prev_tile / tiles_x) * TH);
    }
    if (!ok && tid == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "n"(2 * tc::NCOL));
}

// ---------------------------------------------------------------------------
// Weight gradient: dW[tap][o][c] = sum_cells g[cell][o] x[cell + off(tap)][c]
// (M = output channel, N = input channel, K = cells), per-CTA partial sums
// over a grid-stride set of 16 x 16 tiles; db[o] = sum_cells g[cell][o].
// ---------------------------------------------------------------------------
struct WgradArgs {
    const bf16 *x;   // [N][CINP] layer input
    const bf16 *g;   // [N][COUTP] gradient of the layer's pre-activation output
    float *part;     // [gridDim.x][wg_part_stride]
    int nx, ny, tiles_x, ntiles;
};

template <int CINP, int COUTP>
__global__ void __launch_bounds__(NTHR) wgrad_kernel(WgradArgs a) {
    constexpr int OR = wg_rows(COUTP), MT = OR / 16, NT = CINP / 8, P = MT * NT;
    static_assert(8 % P == 0, "(row block, column block) pairs must divide the 8 warps");
    constexpr int WPP = 8 / P, TPW = (9 + WPP - 1) / WPP;
    constexpr int QI = CINP / 8, QO = COUTP / 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    bf16 *gT = reinterpret_cast<bf16 *>(smem_raw);    // [OR][WG_GS]
    bf16 *xT = gT + OR * WG_GS;                        // [3][CINP][WG_XP]
    float *dbs = reinterpret_cast<float *>(xT + 3 * CINP * WG_XP);   // [8][32]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    const int pair = warp % P, mt = pair / NT, nt = pair % NT, tsel = warp / P;
    const bf16 zero = __float2bfloat16(0.0f);
    for (int i = tid; i < OR * WG_GS; i += NTHR) gT[i] = zero;   // rows >= COUTP stay zero
    float acc[TPW][4];
#pragma unroll
    for (int j = 0; j < TPW; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[j][q] = 0.0f;
    float dbacc = 0.0f;
    const int bo = tid & 31, bseg = tid >> 5;

    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const int ty = tile / a.tiles_x, tx = tile - ty * a.tiles_x;
        const int x0 = tx * TW, y0 = ty * TH;
        __syncthreads();   // the previous tile's operands are consumed
        for (int i = tid; i < TW * TH * QO; i += NTHR) {
            const int cell = i / QO, q = i - cell * QO;
            const int r = cell / TW, c = cell - r * TW;
            const int gy = y0 + r, gx = x0 + c;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (gy < a.ny && gx < a.nx)
                v = reinterpret_cast<const uint4 *>(a.g)[((int64_t)gy * a.nx + gx) * QO + q];
            const bf16 *e = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
            for (int j = 0; j < 8; ++j) gT[(q * 8 + j) * WG_GS + cell] = e[j];
        }
        for (int i = tid; i < HH * HW * QI; i += NTHR) {
            const int cell = i / QI, q = i - cell * QI;
            const int hr = cell / HW, hc = cell - hr * HW;
            const int gy = y0 + hr - 1, gx = x0 + hc - 1;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (gy >= 0 && gy < a.ny && gx >= 0 && gx < a.nx)
                v = reinterpret_cast<const uint4 *>(a.x)[((int64_t)gy * a.nx + gx) * QI + q];
            const bf16 *e = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
            for (int di = 0; di < 3; ++di) {
                const int col = hc - di;
                if (col < 0 || col >= TW) continue;
#pragma unroll
                for (int j = 0; j < 8; ++j) xT[(di * CINP + q * 8 + j) * WG_XP + hr * TW + col] = e[j];
            }
        }
        __syncthreads();
        if (bo < COUTP) {
            float s = 0.0f;
            for (int i = 0; i < 32; ++i) s += __bfloat162float(gT[bo * WG_GS + bseg * 32 + i]);
            dbacc += s;
        }
#pragma unroll 4
        for (int ks = 0; ks < TH; ++ks) {
            const bf16 *ap = gT + (mt * 16 + g) * WG_GS + ks * TW + 2 * t;
            const uint32_t a0 = lds32(ap), a1 = lds32(ap + 8 * WG_GS);
            const uint32_t a2 = lds32(ap + 8), a3 = lds32(ap + 8 * WG_GS + 8);
#pragma unroll
            for (int j = 0; j < TPW; ++j) {
                const int tap = tsel + j * WPP;
                if (tap < 9) {
                    const int dj = tap / 3, di = tap - dj * 3;
                    const bf16 *bp = xT + (di * CINP + nt * 8 + g) * WG_XP + (ks + dj) * TW + 2 * t;
                    mma_bf16(acc[j], a0, a1, a2, a3, lds32(bp), lds32(bp + 8));
                }
            }
        }
    }

    float *part = a.part + (size_t)blockIdx.x * wg_part_stride(CINP, COUTP);
#pragma unroll
    for (int j = 0; j < TPW; ++j) {
        const int tap = tsel + j * WPP;
        if (tap >= 9) continue;
        const int o0 = mt * 16 + g, o1 = o0 + 8, c0 = nt * 8 + 2 * t;
        if (o0 < COUTP) {
            part[((int64_t)tap * COUTP + o0) * CINP + c0] = acc[j][0];
            part[((int64_t)tap * COUTP + o0) * CINP + c0 + 1] = acc[j][1];
        }
        if (o1 < COUTP) {
            part[((int64_t)tap * COUTP + o1) * CINP + c0] = acc[j][2];
            part[((int64_t)tap * COUTP + o1) * CINP + c0 + 1] = acc[j][3];
        }
    }
    dbs[bseg * 32 + bo] = dbacc;
    __syncthreads();
    if (tid < COUTP) {
        float s = 0.0f;
        for (int q = 0; q < 8; ++q) s += dbs[q * 32 + tid];
        part[(int64_t)9 * COUTP * CINP + tid] = s;
    }
}

// ---------------------------------------------------------------------------
// Small kernels: parameter packing, gradient reduction, loss, Adam
// ---------------------------------------------------------------------------
struct Layer {
    int cin, cout, cinp, coutp;
    int64_t w_off, b_off;   // into the flat parameter vector
    bf16 *wf;               // [coutp][kstr(cinp)]
    bf16 *wd;               // [cinp][kstr(coutp)] (layers > 0)
    float *bias;            // [coutp]
};

struct LayerTable {
    Layer l[MAX_LAYERS];
    int n;
};

// blockIdx.y = layer: packed bf16 forward weights, flipped transposed copy and
// the zero-padded FP32 bias.
__global__ void pack_kernel(LayerTable tab, const float *__restrict__ master) {
    const Layer L = tab.l[blockIdx.y];
    const float *W = master + L.w_off;
    const int ksf = kstr(L.cinp), ksd = kstr(L.coutp);
    const int nf = L.coutp * ksf, nd = (blockIdx.y > 0) ? L.cinp * ksd : 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf + nd + L.coutp;
         i += gridDim.x * blockDim.x) {
        if (i < nf) {
            const int o = i / ksf, k = i - o * ksf, tap = k / L.cinp, c = k - tap * L.cinp;
            float v = 0.0f;
            if (tap < 9 && o < L.cout && c < L.cin) v = W[((int64_t)o * L.cin + c) * 9 + tap];
            L.wf[i] = __float2bfloat16_rn(v);
        } else if (i < nf + nd) {
            const int j = i - nf;
            const int c = j / ksd, k = j - c * ksd, tap = k / L.coutp, o = k - tap * L.coutp;
            float v = 0.0f;
            if (tap < 9 && o < L.cout && c < L.cin) v = W[((int64_t)o * L.cin + c) * 9 + (8 - tap)];
            L.wd[j] = __float2bfloat16_rn(v);
        } else {
            const int o = i - nf - nd;
            L.bias[o] = (o < L.cout) ? master[L.b_off + o] : 0.0f;
        }
    }
}

// grad (flat layout of one layer) = (sum over CTAs of the partials) / n_w.
__global__ void grad_reduce_kernel(const float *__restrict__ part, int nblk, int64_t pstride, int cin,
                                   int cout, int cinp, int coutp, const double *__restrict__ stat,
                                   float *__restrict__ grad) {
    const int64_t nw = (int64_t)cout * cin * 9;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nw + cout) return;
    int64_t pi;
    if (i < nw) {
        const int o = (int)(i / ((int64_t)cin * 9));
        const int rem = (int)(i - (int64_t)o * cin * 9);
        const int c = rem / 9, tap = rem - c * 9;
        pi = ((int64_t)tap * coutp + o) * cinp + c;
    } else {
        pi = (int64_t)9 * coutp * cinp + (i - nw);
    }
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += (double)part[(int64_t)b * pstride + pi];
    const double n = stat[0] > 1.0 ? stat[0] : 1.0;
    grad[i] = (float)(s / n);
}

// Block sum of NV doubles (all threads call; thread 0 gets the totals).
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
    __shared__ double sh[NV][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) sh[q][warp] = v[q];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += sh[q][w];
            v[q] = s;
        }
}

// d = (y - target) w; dy = 2 d in channel 0 of [N][8]; partial sum w, sum d^2.
__global__ void __launch_bounds__(RED_THREADS) loss_kernel(int64_t N, const float *__restrict__ y,
                                                           const float *__restrict__ tgt,
                                                           const float *__restrict__ wt,
                                                           bf16 *__restrict__ dy, double *__restrict__ part) {
    double v[2] = {0.0, 0.0};
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        const float w = wt[k];
        const float d = (y[k] - tgt[k]) * w;
        const uint4 o = make_uint4((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(2.0f * d)), 0u, 0u, 0u);
        reinterpret_cast<uint4 *>(dy)[k] = o;
        v[0] += (double)w;
        v[1] += (double)d * (double)d;
    }
    block_sum<2>(v);
    if (threadIdx.x == 0) {
        part[blockIdx.x * NRED + 0] = v[0];
        part[blockIdx.x * NRED + 1] = v[1];
    }
}

// stat[0] = sum w, stat[1] = loss; loss_out (device, may be NULL) = loss.
__global__ void loss_final_kernel(const double *__restrict__ part, int nblk, double *__restrict__ stat,
                                  double *__restrict__ loss_out) {
    double v[2] = {0.0, 0.0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        v[0] += part[b * NRED + 0];
        v[1] += part[b * NRED + 1];
    }
    block_sum<2>(v);
    if (threadIdx.x == 0) {
        stat[0] = v[0];
        stat[1] = v[1] / (v[0] > 1.0 ? v[0] : 1.0);
        if (loss_out) *loss_out = stat[1];
    }
}

// One Adam step (Kingma and Ba, 2015) in FP32; c1, c2 = bias corrections.
__global__ void adam_kernel(int64_t n, float *__restrict__ p, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// ---------------------------------------------------------------------------
// Features and warm start
// ---------------------------------------------------------------------------
// DP offsets from the cell centre in units of l0 (bf16 [N][2]; 0 at void DPs).
__global__ void offsets_kernel(Geo g, const double *__restrict__ pos, const int8_t *__restrict__ mask,
                               bf16 *__restrict__ off) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.N) return;
    const int64_t i = k % g.n[0], j = k / g.n[0];
    double ox = 0.0, oy = 0.0;
    if (mask[k] != 0) {
        const double cx = g.org[0] + ((double)i + 0.5) * g.l0;
        const double cy = g.org[1] + ((double)j + 0.5) * g.l0;
        ox = (pos[k] - cx) / g.l0;
        oy = (pos[g.N + k] - cy) / g.l0;
    }
    off[2 * k] = __double2bfloat16(ox);
    off[2 * k + 1] = __double2bfloat16(oy);
}

// r0 = b - A p; partials: sum r0^2 (non-void), sum dprev^2 (non-void), count
// of non-void DPs, sum r0^2 (all), sum b^2 (all).
__global__ void __launch_bounds__(RED_THREADS) prep_kernel(int64_t N, const int8_t *__restrict__ kind,
                                                           const double *__restrict__ b,
                                                           const double *__restrict__ Ap,
                                                           const double *__restrict__ dprev,
                                                           double *__restrict__ r0, double *__restrict__ part) {
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double r = b[k] - Ap[k];
        r0[k] = r;
        const bool fluid = kind[k] != KIND_VOID;
        if (fluid) {
            v[0] += r * r;
            if (dprev) v[1] += dprev[k] * dprev[k];
            v[2] += 1.0;
        }
        v[3] += r * r;
        v[4] += b[k] * b[k];
    }
    block_sum<5>(v);
    if (threadIdx.x == 0)
        for (int q = 0; q < 5; ++q) part[blockIdx.x * NRED + q] = v[q];
}

// sc[0] = 1/s_r, sc[1] = 1/s_d (0 if s_d = 0), sc[2] = s_out, sc[3] = ||r0||^2,
// sc[4] = ||b||^2 (s_r, s_d: rms over non-void DPs).
__global__ void scales_kernel(const double *__restrict__ part, int nblk, double l0, double *__restrict__ sc) {
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
        for (int q = 0; q < 5; ++q) v[q] += part[b * NRED + q];
    block_sum<5>(v);
    if (threadIdx.x == 0) {
        const double n = v[2];
        const double s_r = n > 0.0 ? sqrt(v[0] / n) : 0.0;
        const double s_d = n > 0.0 ? sqrt(v[1] / n) : 0.0;
        sc[0] = s_r > 0.0 ? 1.0 / s_r : 1.0;
        sc[1] = s_d > 0.0 ? 1.0 / s_d : 0.0;
        sc[2] = s_d > 0.0 ? s_d : (s_r > 0.0 ? s_r : 1.0) * l0 * l0;
        sc[3] = v[3];
        sc[4] = v[4];
    }
}

// Input channels of every DP, bf16 [N][8]; with p_true also the target
// (p_true - p) / s_out and weight 1 on unknown (inner, Neumann) DPs.
__global__ void features_kernel(int64_t N, const int8_t *__restrict__ kind, const bf16 *__restrict__ off,
                                const double *__restrict__ r0, const double *__restrict__ dprev,
                                const double *__restrict__ sc, bf16 *__restrict__ x,
                                const double *__restrict__ p, const double *__restrict__ p_true,
                                float *__restrict__ tgt, float *__restrict__ wt) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int8_t kd = kind[k];
    const bool fluid = kd != KIND_VOID;
    const bf16 zero = __float2bfloat16(0.0f), one = __float2bfloat16(1.0f);
    const bf16 f0 = fluid ? __double2bfloat16(r0[k] * sc[0]) : zero;
    const bf16 f1 = (kd == KIND_INNER) ? one : zero;
    const bf16 f2 = (kd == KIND_DIRICHLET || kd == KIND_NEUMANN) ? one : zero;
    const bf16 f3 = fluid ? zero : one;
    const bf16 f6 = (fluid && dprev) ? __double2bfloat16(dprev[k] * sc[1]) : zero;
    const uint32_t o45 = reinterpret_cast<const uint32_t *>(off)[k];   // channels 4, 5
    reinterpret_cast<uint4 *>(x)[k] = make_uint4(pack2(f0, f1), pack2(f2, f3), o45, pack2(f6, zero));
    if (p_true) {
        const bool unknown = kd == KIND_INNER || kd == KIND_NEUMANN;
        tgt[k] = unknown ? (float)((p_true[k] - p[k]) / sc[2]) : 0.0f;
        wt[k] = unknown ? 1.0f : 0.0f;
    }
}

// e = y s_out on unknown DPs, 0 elsewhere.
__global__ void corr_kernel(int64_t N, const int8_t *__restrict__ kind, const float *__restrict__ y,
                            const double *__restrict__ sc, double *__restrict__ e) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int8_t kd = kind[k];
    e[k] = (kd == KIND_INNER || kd == KIND_NEUMANN) ? (double)y[k] * sc[2] : 0.0;
}

__global__ void __launch_bounds__(RED_THREADS) dots_kernel(int64_t N, const double *__restrict__ r0,
                                                           const double *__restrict__ Ae,
                                                           double *__restrict__ part) {
    double v[2] = {0.0, 0.0};
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        v[0] += r0[k] * Ae[k];
        v[1] += Ae[k] * Ae[k];
    }
    block_sum<2>(v);
    if (threadIdx.x == 0) {
        part[blockIdx.x * NRED + 0] = v[0];
        part[blockIdx.x * NRED + 1] = v[1];
    }
}

// sc[5] = s = <r0, Ae> / <Ae, Ae> (0 if Ae = 0); sc[6] = ||r0 - s Ae||^2.
__global__ void step_kernel(const double *__restrict__ part, int nblk, double *__restrict__ sc) {
    double v[2] = {0.0, 0.0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        v[0] += part[b * NRED + 0];
        v[1] += part[b * NRED + 1];
    }
    block_sum<2>(v);
    if (threadIdx.x == 0) {
        const double s = (v[1] > 0.0 && isfinite(v[0] / v[1])) ? v[0] / v[1] : 0.0;
        sc[5] = s;
        const double rr = sc[3] - s * v[0];
        sc[6] = rr > 0.0 ? rr : 0.0;
    }
}

// d = p - p_in (the increment of a solve).
__global__ void increment_kernel(int64_t N, const double *__restrict__ p, const double *__restrict__ pin,
                                 double *__restrict__ d) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    d[k] = p[k] - pin[k];
}

__global__ void axpy_step_kernel(int64_t N, const double *__restrict__ sc, const double *__restrict__ e,
                                 double *__restrict__ p) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    p[k] += sc[5] * e[k];
}

}  // namespace cnn

cudaError_t cnn_store_offsets(const mcd_stencils *st, const double *pos, const int8_t *mask,
                              cudaStream_t stream) {
    if (st->mesh.dim != 2 || !st->off16) return cudaSuccess;
    const unsigned blocks = (unsigned)((st->geo.N + 255) / 256);
    MCD_KLAUNCH(MCD_K_OTHER, stream, cnn::offsets_kernel<<<blocks, 256, 0, stream>>>(
        st->geo, pos, mask, reinterpret_cast<cnn::bf16 *>(st->off16)));
    return cudaGetLastError();
}

}  // namespace mcd

using namespace mcd;
using namespace mcd::cnn;

struct mcd_net {
    int c_in, width, layers;
    int64_t n_params;
    float *master = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    LayerTable tab{};
    int step = 0;
    // scratch, sized for `cap` cells
    int64_t cap = 0;
    bf16 *act[MAX_LAYERS] = {};   // hidden activations [cap][32]
    bf16 *ga = nullptr, *gb = nullptr;   // gradient ping-pong [cap][32]
    bf16 *dy = nullptr;           // [cap][8]
    bf16 *x = nullptr;            // features [cap][8]
    float *y = nullptr;           // [cap]
    double *r0 = nullptr, *ap = nullptr, *e = nullptr;   // [cap]
    double *pin = nullptr;        // [cap] guess of the last solve (increment)
    double *part = nullptr;       // [RED_BLOCKS][NRED]
    double *sc = nullptr;         // [8]
    double *stat = nullptr;       // [4]
    int *tc_err = nullptr;        // set by a tensor-core convolution whose MMA wait gave up
    float *wpart = nullptr;       // wgrad partials
    int wg_blocks = 0;
};

namespace {

int64_t layer_params(int cin, int cout) { return (int64_t)cout * cin * 9 + cout; }

void free_scratch(mcd_net *n) {
    for (int l = 0; l < MAX_LAYERS; ++l) {
        cudaFree(n->act[l]);
        n->act[l] = nullptr;
    }
    cudaFree(n->ga);
    cudaFree(n->gb);
    cudaFree(n->dy);
    cudaFree(n->x);
    cudaFree(n->y);
    cudaFree(n->r0);
    cudaFree(n->ap);
    cudaFree(n->e);
    cudaFree(n->pin);
    n->ga = n->gb = n->dy = n->x = nullptr;
    n->y = nullptr;
    n->r0 = n->ap = n->e = n->pin = nullptr;
    n->cap = 0;
}

mcd_status ensure_scratch(mcd_net *n, int64_t N) {
    if (N <= n->cap) return MCD_OK;
    free_scratch(n);
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    for (int l = 0; l + 1 < n->layers; ++l) chk(cudaMalloc(&n->act[l], (size_t)N * WIDTH * sizeof(bf16)));
    chk(cudaMalloc(&n->ga, (size_t)N * WIDTH * sizeof(bf16)));
    chk(cudaMalloc(&n->gb, (size_t)N * WIDTH * sizeof(bf16)));
    chk(cudaMalloc(&n->dy, (size_t)N * FEAT * sizeof(bf16)));
    chk(cudaMalloc(&n->x, (size_t)N * FEAT * sizeof(bf16)));
    chk(cudaMalloc(&n->y, (size_t)N * sizeof(float)));
    chk(cudaMalloc(&n->r0, (size_t)N * sizeof(double)));
    chk(cudaMalloc(&n->ap, (size_t)N * sizeof(double)));
    chk(cudaMalloc(&n->e, (size_t)N * sizeof(double)));
    chk(cudaMalloc(&n->pin, (size_t)N * sizeof(double)));
    if (e != cudaSuccess) {
        free_scratch(n);
        cudaGetLastError();
        set_error(std::string("network scratch allocation: ") + cudaGetErrorString(e));
        return MCD_ENOMEM;
    }
    n->cap = N;
    return MCD_OK;
}

template <int CINP, int COUTP, int EPI>
mcd_status launch_conv(const ConvArgs &a, cudaStream_t s) {
    constexpr size_t sm = conv_smem(CINP, COUTP);
    static bool attr = false;
    if (!attr) {
        MCD_CUDA_TRY(cudaFuncSetAttribute(conv_kernel<CINP, COUTP, EPI>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        attr = true;
    }
    const dim3 grid((unsigned)((a.nx + TW - 1) / TW), (unsigned)((a.ny + TH - 1) / TH));
    MCD_KLAUNCH(MCD_K_CNN, s, conv_kernel<CINP, COUTP, EPI><<<grid, NTHR, sm, s>>>(a));
    MCD_LAUNCH_CHECK();
    return MCD_OK;
}

// Hidden-layer convolution on the tcgen05 tensor cores (forward with bias and
// ReLU, or the input-gradient pass gated by the forward activation).
template <int EPI>
mcd_status launch_conv_tc(const ConvArgs &a, int *err, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        MCD_CUDA_TRY(cudaFuncSetAttribute(conv_tc_kernel<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)tc::SMEM));
        // prefer the whole unified L1 as shared memory, so that several
        // CTAs fit on one SM
        MCD_CUDA_TRY(cudaFuncSetAttribute(conv_tc_kernel<EPI>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          (int)cudaSharedmemCarveoutMaxShared));
        attr = true;
    }
    static int slots = 0;
    if (!slots) {
        // resident CTAs per SM from the SM's shared memory, registers and
        // tensor-memory columns (512, 2 x 64 per CTA)
        int dev = 0, sms = 0, smem_sm = 0, smem_res = 0, regs_sm = 0;
        cudaFuncAttributes fa;
        MCD_CUDA_TRY(cudaGetDevice(&dev));
        MCD_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        MCD_CUDA_TRY(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        MCD_CUDA_TRY(cudaDeviceGetAttribute(&smem_res, cudaDevAttrReservedSharedMemoryPerBlock, dev));
        MCD_CUDA_TRY(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
        MCD_CUDA_TRY(cudaFuncGetAttributes(&fa, conv_tc_kernel<EPI>));
        const int by_smem = smem_sm / (int)(tc::SMEM + fa.sharedSizeBytes + smem_res);
        const int by_regs = regs_sm / std::max(1, fa.numRegs * 256);
        const int by_tmem = 512 / (2 * tc::NCOL);
        slots = std::max(1, std::min(std::min(by_smem, by_regs), by_tmem)) * std::max(1, sms);
    }
    const int ntiles = ((a.nx + TW - 1) / TW) * ((a.ny + TH - 1) / TH);
    const unsigned grid = (unsigned)std::min(ntiles, slots);
    MCD_KLAUNCH(MCD_K_CNN, s, conv_tc_kernel<EPI><<<grid, 256, tc::SMEM, s>>>(a, err));
    MCD_LAUNCH_CHECK();
    return MCD_OK;
}

template <int CINP, int COUTP>
mcd_status launch_wgrad(mcd_net *n, const bf16 *x, const bf16 *g, int nx, int ny, cudaStream_t s) {
    constexpr size_t sm = wgrad_smem(CINP, COUTP);
    static bool attr = false;
    if (!attr) {
        MCD_CUDA_TRY(cudaFuncSetAttribute(wgrad_kernel<CINP, COUTP>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        attr = true;
    }
    WgradArgs a;
    a.x = x;
    a.g = g;
    a.part = n->wpart;
    a.nx = nx;
    a.ny = ny;
    a.tiles_x = (nx + TW - 1) / TW;
    a.ntiles = a.tiles_x * ((ny + TH - 1) / TH);
    MCD_KLAUNCH(MCD_K_CNN, s, wgrad_kernel<CINP, COUTP><<<n->wg_blocks, NTHR, sm, s>>>(a));
    MCD_LAUNCH_CHECK();
    return MCD_OK;
}

mcd_status pack(mcd_net *n, cudaStream_t s) {
    MCD_KLAUNCH(MCD_K_CNN, s, pack_kernel<<<dim3(16, n->layers), 256, 0, s>>>(n->tab, n->master));
    MCD_LAUNCH_CHECK();
    return MCD_OK;
}

// Forward pass of the features x ([N][8]) into n->y; hidden activations kept.
mcd_status forward(mcd_net *n, const bf16 *x, int nx, int ny, float *y, cudaStream_t s) {
    const int L = n->layers;
    ConvArgs a{};
    a.nx = nx;
    a.ny = ny;
    for (int l = 0; l < L; ++l) {
        const Layer &ly = n->tab.l[l];
        a.in = (l == 0) ? x : n->act[l - 1];
        a.w = ly.wf;
        a.bias = ly.bias;
        mcd_status st;
        if (l + 1 < L) {
            a.out = n->act[l];
            st = (l == 0) ? launch_conv<FEAT, WIDTH, EPI_RELU>(a, s) : launch_conv_tc<EPI_RELU>(a, n->tc_err, s);
        } else {
            a.out32 = y;
            st = (l == 0) ? launch_conv<FEAT, FEAT, EPI_LAST>(a, s) : launch_conv<WIDTH, FEAT, EPI_LAST>(a, s);
        }
        if (st != MCD_OK) return st;
    }
    return MCD_OK;
}

unsigned red_blocks(int64_t N) {
    const int64_t b = (N + RED_THREADS - 1) / RED_THREADS;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, RED_BLOCKS));
}

mcd_status check_grid(const mcd_net *n, int nx, int ny) {
    MCD_CHECK_ARG(n, "NULL network");
    MCD_CHECK_ARG(nx > 0 && ny > 0, "grid sizes must be positive");
    MCD_CHECK_ARG((ny + TH - 1) / TH <= 65535, "n_y too large for the tile grid");
    return MCD_OK;
}

// features of (b, p, dprev) into n->x (and target / weight with p_true).
mcd_status make_features(mcd_net *n, const mcd_stencils *st, const double *b, const double *p,
                         const double *dprev, const double *p_true, bf16 *x, float *tgt, float *wt,
                         cudaStream_t s) {
    const int64_t N = st->geo.N;
    mcd_status r = mcd_apply_laplacian(st, p, n->ap, MCD_DT_F64, s);
    if (r != MCD_OK) return r;
    const unsigned rb = red_blocks(N);
    MCD_KLAUNCH(MCD_K_CNN, s, prep_kernel<<<rb, RED_THREADS, 0, s>>>(N, st->kind, b, n->ap, dprev, n->r0, n->part));
    MCD_LAUNCH_CHECK();
    MCD_KLAUNCH(MCD_K_CNN, s, scales_kernel<<<1, 256, 0, s>>>(n->part, (int)rb, st->geo.l0, n->sc));
    MCD_LAUNCH_CHECK();
    const unsigned eb = (unsigned)((N + 255) / 256);
    MCD_KLAUNCH(MCD_K_CNN, s, features_kernel<<<eb, 256, 0, s>>>(N, st->kind, reinterpret_cast<const bf16 *>(st->off16),
                                                                n->r0, dprev, n->sc, x, p, p_true, tgt, wt));
    MCD_LAUNCH_CHECK();
    return MCD_OK;
}

mcd_status check_stencils(const mcd_stencils *st) {
    MCD_CHECK_ARG(st, "NULL stencil handle");
    if (st->mesh.dim != 2 || !st->off16) {
        set_error("the network warm start is 2D only");
        return MCD_ENOTSUP;
    }
    return MCD_OK;
}

}  // namespace

namespace mcd {

// Warm start used by mcd_solve_pressure: p <- p + s e (b: assembled RHS).
// host_sc (8 doubles, may be NULL; synchronises the stream when given):
// 0 1/s_r, 1 1/s_d, 2 s_out, 3 ||r0||^2, 4 ||b||^2, 5 step s, 6 ||r after||^2.
mcd_status net_warm_start(const mcd_net *cnet, const mcd_stencils *st, const double *b, const double *dprev,
                          double *p, double *host_sc, cudaStream_t s) {
    mcd_net *n = const_cast<mcd_net *>(cnet);
    mcd_status r = check_stencils(st);
    if (r != MCD_OK) return r;
    const int nx = st->mesh.n[0], ny = st->mesh.n[1];
    r = check_grid(n, nx, ny);
    if (r != MCD_OK) return r;
    const int64_t N = st->geo.N;
    r = ensure_scratch(n, N);
    if (r != MCD_OK) return r;
    r = make_features(n, st, b, p, dprev, nullptr, n->x, nullptr, nullptr, s);
    if (r != MCD_OK) return r;
    r = forward(n, n->x, nx, ny, n->y, s);
    if (r != MCD_OK) return r;
    const unsigned eb = (unsigned)((N + 255) / 256);
    MCD_KLAUNCH(MCD_K_CNN, s, corr_kernel<<<eb, 256, 0, s>>>(N, st->kind, n->y, n->sc, n->e));
    MCD_LAUNCH_CHECK();
    r = mcd_apply_laplacian(st, n->e, n->ap, MCD_DT_F64, s);
    if (r != MCD_OK) return r;
    const unsigned rb = red_blocks(N);
    MCD_KLAUNCH(MCD_K_CNN, s, dots_kernel<<<rb, RED_THREADS, 0, s>>>(N, n->r0, n->ap, n->part));
    MCD_LAUNCH_CHECK();
    MCD_KLAUNCH(MCD_K_CNN, s, step_kernel<<<1, 256, 0, s>>>(n->part, (int)rb, n->sc));
    MCD_LAUNCH_CHECK();
    MCD_KLAUNCH(MCD_K_CNN, s, axpy_step_kernel<<<eb, 256, 0, s>>>(N, n->sc, n->e, p));
    MCD_LAUNCH_CHECK();
    if (host_sc) {
        MCD_CUDA_TRY(cudaMemcpyAsync(host_sc, n->sc, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
        MCD_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return MCD_OK;
}

// Keep the guess of a solve (before its Dirichlet values and warm start).
mcd_status net_save_guess(const mcd_net *cnet, const mcd_stencils *st, const double *p, cudaStream_t s) {
    mcd_net *n = const_cast<mcd_net *>(cnet);
    mcd_status r = ensure_scratch(n, st->geo.N);
    if (r != MCD_OK) return r;
    MCD_CUDA_TRY(cudaMemcpyAsync(n->pin, p, st->geo.N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return MCD_OK;
}

// dprev = p - (the saved guess): the increment the next warm start reads.
mcd_status net_store_increment(const mcd_net *cnet, const mcd_stencils *st, const double *p, double *dprev,
                               cudaStream_t s) {
    const int64_t N = st->geo.N;
    const unsigned eb = (unsigned)((N + 255) / 256);
    MCD_KLAUNCH(MCD_K_CNN, s, increment_kernel<<<eb, 256, 0, s>>>(N, p, cnet->pin, dprev));
    MCD_LAUNCH_CHECK();
    return MCD_OK;
}

}  // namespace mcd

extern "C" int64_t mcd_net_param_count(int c_in, int width, int layers) {
    if (c_in < 1 || c_in > FEAT || width != WIDTH || layers < 2 || layers > MAX_LAYERS) return -1;
    int64_t n = layer_params(c_in, width) + layer_params(width, 1);
    n += (int64_t)(layers - 2) * layer_params(width, width);
    return n;
}

extern "C" mcd_status mcd_net_create(int c_in, int width, int layers, const float *params,
                                     int64_t n_params, mcd_net **out) {
    MCD_CHECK_ARG(out && params, "NULL argument");
    const int64_t want = mcd_net_param_count(c_in, width, layers);
    if (want < 0) {
        set_error("unsupported network shape (c_in in [1, 8], width 32, layers in [2, 8])");
        return MCD_ENOTSUP;
    }
    MCD_CHECK_ARG(n_params == want, "n_params does not match the network shape");
    mcd_net *n = new mcd_net();
    n->c_in = c_in;
    n->width = width;
    n->layers = layers;
    n->n_params = want;
    n->tab.n = layers;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    chk(cudaMalloc(&n->master, want * sizeof(float)));
    chk(cudaMalloc(&n->grad, want * sizeof(float)));
    chk(cudaMalloc(&n->m, want * sizeof(float)));
    chk(cudaMalloc(&n->v, want * sizeof(float)));
    int64_t at = 0;
    for (int l = 0; l < layers; ++l) {
        Layer &L = n->tab.l[l];
        L.cin = (l == 0) ? c_in : width;
        L.cout = (l + 1 == layers) ? 1 : width;
        L.cinp = (l == 0) ? FEAT : WIDTH;
        L.coutp = (l + 1 == layers) ? FEAT : WIDTH;
        L.w_off = at;
        L.b_off = at + (int64_t)L.cout * L.cin * 9;
        at += layer_params(L.cin, L.cout);
        chk(cudaMalloc(&L.wf, (size_t)L.coutp * kstr(L.cinp) * sizeof(bf16)));
        if (l > 0) chk(cudaMalloc(&L.wd, (size_t)L.cinp * kstr(L.coutp) * sizeof(bf16)));
        chk(cudaMalloc(&L.bias, (size_t)L.coutp * sizeof(float)));
    }
    int dev = 0, sms = 0;
    chk(cudaGetDevice(&dev));
    chk(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    n->wg_blocks = std::max(1, sms) * 2;
    chk(cudaMalloc(&n->wpart, (size_t)n->wg_blocks * wg_part_stride(WIDTH, WIDTH) * sizeof(float)));
    chk(cudaMalloc(&n->part, (size_t)RED_BLOCKS * NRED * sizeof(double)));
    chk(cudaMalloc(&n->sc, 8 * sizeof(double)));
    chk(cudaMalloc(&n->stat, 4 * sizeof(double)));
    chk(cudaMalloc(&n->tc_err, sizeof(int)));
    if (e == cudaSuccess) chk(cudaMemset(n->tc_err, 0, sizeof(int)));
    if (e == cudaSuccess) chk(cudaMemcpy(n->master, params, want * sizeof(float), cudaMemcpyHostToDevice));
    if (e == cudaSuccess) chk(cudaMemset(n->grad, 0, want * sizeof(float)));
    if (e == cudaSuccess) chk(cudaMemset(n->m, 0, want * sizeof(float)));
    if (e == cudaSuccess) chk(cudaMemset(n->v, 0, want * sizeof(float)));
    if (e != cudaSuccess) {
        cudaGetLastError();
        mcd_net_destroy(n);
        set_error(std::string("network allocation: ") + cudaGetErrorString(e));
        return MCD_ENOMEM;
    }
    mcd_status s = pack(n, nullptr);
    if (s != MCD_OK) {
        mcd_net_destroy(n);
        return s;
    }
    MCD_CUDA_TRY(cudaDeviceSynchronize());
    *out = n;
    return MCD_OK;
}

extern "C" void mcd_net_destroy(mcd_net *n) {
    if (!n) return;
    free_scratch(n);
    for (int l = 0; l < MAX_LAYERS; ++l) {
        cudaFree(n->tab.l[l].wf);
        cudaFree(n->tab.l[l].wd);
        cudaFree(n->tab.l[l].bias);
    }
    cudaFree(n->master);
    cudaFree(n->grad);
    cudaFree(n->m);
    cudaFree(n->v);
    cudaFree(n->wpart);
    cudaFree(n->part);
    cudaFree(n->sc);
    cudaFree(n->stat);
    cudaFree(n->tc_err);
    delete n;
}

extern "C" mcd_status mcd_net_read(const mcd_net *n, int which, float *host_out, int64_t count) {
    MCD_CHECK_ARG(n && host_out, "NULL argument");
    MCD_CHECK_ARG(count == n->n_params, "count must equal the parameter count");
    const float *src = nullptr;
    if (which == MCD_NET_PARAMS) src = n->master;
    else if (which == MCD_NET_GRADS) src = n->grad;
    else if (which == MCD_NET_ADAM_M) src = n->m;
    else if (which == MCD_NET_ADAM_V) src = n->v;
    MCD_CHECK_ARG(src, "unknown array");
    MCD_CUDA_TRY(cudaDeviceSynchronize());
    MCD_CUDA_TRY(cudaMemcpy(host_out, src, count * sizeof(float), cudaMemcpyDeviceToHost));
    int tc_err = 0;
    MCD_CUDA_TRY(cudaMemcpy(&tc_err, n->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (tc_err) {
        set_error("a tensor-core convolution gave up waiting for its MMAs; results since are invalid");
        return MCD_ETIMEOUT;
    }
    return MCD_OK;
}

extern "C" mcd_status mcd_net_features(mcd_net *n, const mcd_stencils *st, const double *b_dev,
                                       const double *p_dev, const double *dprev_dev,
                                       const double *p_true_dev, uint16_t *x_dev, float *target_dev,
                                       float *weight_dev, mcd_stream_t stream) {
    MCD_CHECK_ARG(n && b_dev && p_dev && x_dev, "NULL argument");
    MCD_CHECK_ARG(!p_true_dev || (target_dev && weight_dev), "target and weight outputs are required with p_true");
    mcd_status r = check_stencils(st);
    if (r != MCD_OK) return r;
    r = ensure_scratch(n, st->geo.N);
    if (r != MCD_OK) return r;
    return make_features(n, st, b_dev, p_dev, dprev_dev, p_true_dev, reinterpret_cast<bf16 *>(x_dev),
                         target_dev, weight_dev, stream);
}

extern "C" mcd_status mcd_net_forward(mcd_net *n, const uint16_t *x_dev, int nx, int ny, float *y_dev,
                                      mcd_stream_t stream) {
    mcd_status r = check_grid(n, nx, ny);
    if (r != MCD_OK) return r;
    MCD_CHECK_ARG(x_dev && y_dev, "NULL argument");
    r = ensure_scratch(n, (int64_t)nx * ny);
    if (r != MCD_OK) return r;
    return forward(n, reinterpret_cast<const bf16 *>(x_dev), nx, ny, y_dev, stream);
}

extern "C" mcd_status mcd_net_train_step(mcd_net *n, const uint16_t *x_dev, const float *target_dev,
                                         const float *weight_dev, int nx, int ny, float lr,
                                         double *loss_dev, mcd_stream_t stream) {
    mcd_status r = check_grid(n, nx, ny);
    if (r != MCD_OK) return r;
    MCD_CHECK_ARG(x_dev && target_dev && weight_dev, "NULL argument");
    MCD_CHECK_ARG(lr > 0.0f && std::isfinite(lr), "lr must be positive");
    const int64_t N = (int64_t)nx * ny;
    r = ensure_scratch(n, N);
    if (r != MCD_OK) return r;
    cudaStream_t s = stream;
    const bf16 *x = reinterpret_cast<const bf16 *>(x_dev);
    r = forward(n, x, nx, ny, n->y, s);
    if (r != MCD_OK) return r;
    const unsigned rb = red_blocks(N);
    MCD_KLAUNCH(MCD_K_CNN, s, loss_kernel<<<rb, RED_THREADS, 0, s>>>(N, n->y, target_dev, weight_dev, n->dy, n->part));
    MCD_LAUNCH_CHECK();
    MCD_KLAUNCH(MCD_K_CNN, s, loss_final_kernel<<<1, 256, 0, s>>>(n->part, (int)rb, n->stat, loss_dev));
    MCD_LAUNCH_CHECK();
    // backward: g holds the gradient of the current layer's pre-activation
    // output (channels-last); the input gradient of layer l > 0 is gated by
    // the ReLU of layer l - 1 (its forward output act[l-1] > 0).
    const int L = n->layers;
    const bf16 *g = n->dy;
    for (int l = L - 1; l >= 0; --l) {
        const Layer &ly = n->tab.l[l];
        const bf16 *xin = (l == 0) ? x : n->act[l - 1];
        if (l == 0) r = (l + 1 == L) ? launch_wgrad<FEAT, FEAT>(n, xin, g, nx, ny, s)
                                     : launch_wgrad<FEAT, WIDTH>(n, xin, g, nx, ny, s);
        else r = (l + 1 == L) ? launch_wgrad<WIDTH, FEAT>(n, xin, g, nx, ny, s)
                              : launch_wgrad<WIDTH, WIDTH>(n, xin, g, nx, ny, s);
        if (r != MCD_OK) return r;
        const int64_t nl = layer_params(ly.cin, ly.cout);
        MCD_KLAUNCH(MCD_K_CNN, s, grad_reduce_kernel<<<(unsigned)((nl + 255) / 256), 256, 0, s>>>(
            n->wpart, n->wg_blocks, wg_part_stride(ly.cinp, ly.coutp), ly.cin, ly.cout, ly.cinp, ly.coutp,
            n->stat, n->grad + ly.w_off));
        MCD_LAUNCH_CHECK();
        if (l > 0) {
            bf16 *gout = (g == n->ga) ? n->gb : n->ga;
            ConvArgs a{};
            a.in = g;
            a.w = ly.wd;
            a.gate = n->act[l - 1];
            a.out = gout;
            a.nx = nx;
            a.ny = ny;
            r = (l + 1 == L) ? launch_conv<FEAT, WIDTH, EPI_DGRAD>(a, s)
                             : launch_conv_tc<EPI_DGRAD>(a, n->tc_err, s);
            if (r != MCD_OK) return r;
            g = gout;
        }
    }
    n->step += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 / (1.0 - std::pow(b1, n->step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow(b2, n->step)));
    MCD_KLAUNCH(MCD_K_CNN, s, adam_kernel<<<(unsigned)((n->n_params + 255) / 256), 256, 0, s>>>(
        n->n_params, n->master, n->grad, n->m, n->v, lr, (float)b1, (float)b2, 1e-8f, c1, c2));
    MCD_LAUNCH_CHECK();
    return pack(n, s);
}

extern "C" mcd_status mcd_net_warm_start(mcd_net *n, const mcd_stencils *st, const double *b_dev,
                                         const double *dprev_dev, double *p_dev, double *stats,
                                         mcd_stream_t stream) {
    MCD_CHECK_ARG(n && b_dev && p_dev, "NULL argument");
    double h[8];
    mcd_status r = net_warm_start(n, st, b_dev, dprev_dev, p_dev, stats ? h : nullptr, stream);
    if (r != MCD_OK) return r;
    if (stats) {
        const double bb = h[4];
        stats[0] = bb > 0.0 ? std::sqrt(h[3] / bb) : 0.0;
        stats[1] = bb > 0.0 ? std::sqrt(h[6] / bb) : 0.0;
        stats[2] = h[5];
    }
    return MCD_OK;
}
