// The 3D U-Net of the learned warm start, with hand-written forward,
// backward and Adam kernels.  The 3x3x3 convolutions (forward, data gradient
// and weight gradient) are implicit GEMMs on the tensor cores: BF16 operands,
// FP32 accumulation (mma.sync m16n8k16); everything else is FP32 elementwise
// work.  Sums run in a fixed order (no atomics), so results are bitwise
// reproducible.
//
// Architecture (widths 16-32-48-64, "same" zero padding, ReLU after every
// 3x3x3 convolution, 2x2x2 average pooling, nearest upsampling, the skip
// joined after the upsampled channels):
//   L0  cin -> 16, L1 16 -> 16 (e1)          | level 1 (full grid)
//   L2  16 -> 32,  L3 32 -> 32 (e2)          | level 2 (pool e1)
//   L4  32 -> 48,  L5 48 -> 48 (e3)          | level 3 (pool e2)
//   L6  48 -> 64,  L7 64 -> 64               | level 4 (pool e3)
//   L8  [up L7, e3] 112 -> 48, L9 48 -> 48   | level 3
//   L10 [up L9, e2]  80 -> 32, L11 32 -> 32  | level 2
//   L12 [up L11, e1] 48 -> 16, L13 16 -> 16  | level 1
//   L14 16 -> cout (1x1, no ReLU)
// Mixed precision: weights, the input, every stored activation and every
// gradient signal entering a convolution's backward pass are BF16 (round to
// nearest even); biases, the output, the loss and its gradient are FP32.
// Activations are stored channels-last ([voxel][channel]); the public
// tensors are FP32 [channel][D][H][W] (W fastest) with D, H, W multiples of 8.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <string>
#include <vector>

#include "ht.h"

namespace {

typedef __nv_bfloat16 bf16;

constexpr int kLayers = 15;
constexpr int kW1 = 16, kW2 = 32, kW3 = 48, kW4 = 64;
constexpr int kThreads = 256;      // 8 warps
constexpr int kConvVox = 128;      // voxels per CTA of the convolution (16 per warp)
constexpr int kWgVox = 64;         // voxels per staged block of the weight gradient
constexpr int kWgSplit = 24;       // K splits of the weight gradient (partial sums)

struct Vol {
    int D, H, W;
    __host__ __device__ long long n() const { return (long long)D * H * W; }
};

// ---------------------------------------------------------------------------
// tensor-core primitives (PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], const void* smem_row) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem_row);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

__device__ __forceinline__ void ldsm_x2_trans(uint32_t& r0, uint32_t& r1, const void* smem_row) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem_row);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}

__device__ __forceinline__ uint32_t ld_pair(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// ---------------------------------------------------------------------------
// 3x3x3 convolution as an implicit GEMM (forward and data gradient)
//   out[v][n0 + j] = bias + sum_t sum_k in[v + d_t][k] W[t][n0 + j][k]
// in: BF16 [V][ld_in] (K channels used, K a multiple of 16); W: BF16
// [27][Nout][K]; a CTA of 8 warps takes 128 voxels, each warp 16 voxels and
// NT * 8 output channels.  The weights of one 16-channel K chunk (all taps)
// are staged in shared memory; the A fragments come from global memory
// (they are reused across the 27 taps through L1).  flip: tap t reads the
// neighbour at -d_t (the data gradient, with W transposed:
// g_in[v][ci] = sum_t sum_co W[t][co][ci] s[v - d_t][co]).
// ---------------------------------------------------------------------------
template <int NT>
__global__ void __launch_bounds__(kThreads) conv3_kernel(const bf16* __restrict__ in, const int ld_in, const int K,
                                                        const bf16* __restrict__ Wt, const int Nout, const int n0,
                                                        const float* __restrict__ bias, bf16* __restrict__ out_b,
                                                        float* __restrict__ out_f, const int ld_out,
                                                        const int relu, const Vol v, const int flip) {
    extern __shared__ __align__(16) unsigned char conv_smem_raw[];
    bf16* ws = reinterpret_cast<bf16*>(conv_smem_raw);      // [27][NT*8][24] (16 used, padded rows)
    constexpr int NC = NT * 8, ROW = 24;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tig = lane & 3;
    const long long V = v.n();
    const long long vbase = (long long)blockIdx.x * kConvVox + warp * 16;
    // the thread's two voxels (rows g and g + 8 of the warp tile)
    long long vv[2];
    int vz[2], vy[2], vx[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        vv[h] = vbase + g + 8 * h;
        const long long q = vv[h] < V ? vv[h] : 0;
        vx[h] = (int)(q % v.W);
        vy[h] = (int)((q / v.W) % v.H);
        vz[h] = (int)(q / ((long long)v.W * v.H));
    }
    float acc[NT][4];
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
    const long long HW = (long long)v.H * v.W;
    for (int k0 = 0; k0 < K; k0 += 16) {
        __syncthreads();
        // stage W[t][n0 .. n0 + NC)[k0 .. k0 + 16) as 16-byte chunks
        for (int c = threadIdx.x; c < 27 * NC * 2; c += kThreads) {
            const int half = c & 1, row = c >> 1;       // row = t * NC + j
            const int t = row / NC, j = row % NC;
            const uint4 val = *reinterpret_cast<const uint4*>(Wt + ((long long)t * Nout + n0 + j) * K + k0 + 8 * half);
            *reinterpret_cast<uint4*>(ws + row * ROW + 8 * half) = val;
        }
        __syncthreads();
        for (int t = 0; t < 27; ++t) {
            int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
            if (flip) { dz = -dz; dy = -dy; dx = -dx; }
            uint32_t a[4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int z = vz[h] + dz, y = vy[h] + dy, x = vx[h] + dx;
                const bool ok = vv[h] < V && z >= 0 && z < v.D && y >= 0 && y < v.H && x >= 0 && x < v.W;
                const long long nb = (long long)z * HW + (long long)y * v.W + x;
                const bf16* p = in + (ok ? nb : 0) * ld_in + k0 + 2 * tig;
                a[h] = ok ? ld_pair(p) : 0u;          // rows g / g + 8, columns 2 tig, 2 tig + 1
                a[2 + h] = ok ? ld_pair(p + 8) : 0u;  // columns 2 tig + 8, + 9
            }
            const bf16* wt = ws + (t * NC + g) * ROW + 2 * tig;
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const uint32_t b0 = *reinterpret_cast<const uint32_t*>(wt + j * 8 * ROW);
                const uint32_t b1 = *reinterpret_cast<const uint32_t*>(wt + j * 8 * ROW + 8);
                mma_bf16(acc[j], a, b0, b1);
            }
        }
    }
    // epilogue: rows g, g + 8; columns j * 8 + 2 tig, + 1
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (vv[h] >= V) continue;
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const int col = j * 8 + 2 * tig;
            float o0 = acc[j][2 * h], o1 = acc[j][2 * h + 1];
            if (bias) { o0 += bias[n0 + col]; o1 += bias[n0 + col + 1]; }
            if (relu) { o0 = fmaxf(o0, 0.0f); o1 = fmaxf(o1, 0.0f); }
            if (out_b) {
                __nv_bfloat162 pr = __floats2bfloat162_rn(o0, o1);
                *reinterpret_cast<__nv_bfloat162*>(out_b + vv[h] * ld_out + n0 + col) = pr;
            } else {
                *reinterpret_cast<float2*>(out_f + vv[h] * ld_out + n0 + col) = make_float2(o0, o1);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Weight gradient of a 3x3x3 convolution on the tensor cores:
//   dW[t][co][ci] = sum_v s[v][co] in[v + d_t][ci]
// (M = co, N = ci, K = voxels).  A CTA takes one tap and a range of voxel
// blocks; each block of 64 voxels stages s [64][Cout] and the tap-shifted
// input [64][Cin] in shared memory, and ldmatrix.trans turns both into
// fragments (A = s^T, B = in).  Every warp owns some (16 x 8) output tiles;
// the CTA's partial sums go to part[split][t][co][ci], reduced in a fixed
// order by wgrad_reduce_kernel.
// ---------------------------------------------------------------------------
constexpr int kWgTiles = 7;   // output tiles per warp at most: (64 / 16) * (112 / 8) / 8 = 7

__global__ void __launch_bounds__(kThreads) wgrad_kernel(const bf16* __restrict__ sig, const int Cout,
                                                        const bf16* __restrict__ in, const int ld_in, const int Cin,
                                                        const Vol v, float* __restrict__ part, const int nsplit) {
    extern __shared__ __align__(16) unsigned char wg_smem[];
    const int lds = Cout + 8, ldi = Cin + 8;                  // padded rows (16 bytes)
    bf16* S = reinterpret_cast<bf16*>(wg_smem);               // [64][Cout + 8]
    bf16* I = S + kWgVox * lds;                               // [64][Cin + 8]
    const int t = blockIdx.y, split = blockIdx.x;
    const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long V = v.n(), HW = (long long)v.H * v.W;
    const long long nblk = (V + kWgVox - 1) / kWgVox;
    const long long b0 = nblk * split / nsplit, b1 = nblk * (split + 1) / nsplit;
    const int mt_n = Cout / 16, nt_n = Cin / 8, tiles = mt_n * nt_n;
    float acc[kWgTiles][4];
#pragma unroll
    for (int i = 0; i < kWgTiles; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.0f;
    for (long long blk = b0; blk < b1; ++blk) {
        const long long v0 = blk * kWgVox;
        __syncthreads();
        // stage the signal rows and the tap-shifted input rows (16-byte chunks)
        const int cs = Cout / 8, ci8 = Cin / 8;
        for (int c = threadIdx.x; c < kWgVox * (cs + ci8); c += kThreads) {
            const bool is_s = c < kWgVox * cs;
            const int cc = is_s ? c : c - kWgVox * cs;
            const int per = is_s ? cs : ci8;
            const int r = cc / per, q = cc % per;
            const long long vox = v0 + r;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (vox < V) {
                if (is_s) {
                    val = *reinterpret_cast<const uint4*>(sig + vox * Cout + 8 * q);
                } else {
                    const int x = (int)(vox % v.W) + dx, y = (int)((vox / v.W) % v.H) + dy,
                              z = (int)(vox / HW) + dz;
                    if (z >= 0 && z < v.D && y >= 0 && y < v.H && x >= 0 && x < v.W)
                        val = *reinterpret_cast<const uint4*>(in + ((long long)z * HW + (long long)y * v.W + x) *
                                                                       ld_in + 8 * q);
                }
            }
            bf16* dst = is_s ? S + r * lds + 8 * q : I + r * ldi + 8 * q;
            *reinterpret_cast<uint4*>(dst) = val;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < kWgVox / 16; ++ks) {
            const int kr = ks * 16;
#pragma unroll
            for (int i = 0; i < kWgTiles; ++i) {
                const int tile = warp + 8 * i;
                if (tile >= tiles) break;
                const int mt = tile % mt_n, nt = tile / mt_n;
                // A = s^T: matrices (k 0-7, m 0-7), (k 0-7, m 8-15), (k 8-15, m 0-7), (k 8-15, m 8-15)
                uint32_t a[4];
                const int arow = kr + (lane & 7) + ((lane >> 4) << 3);
                const int acol = mt * 16 + (((lane >> 3) & 1) << 3);
                ldsm_x4_trans(a, S + arow * lds + acol);
                // B = in: matrices (k 0-7, n), (k 8-15, n)
                uint32_t bb0, bb1;
                const int brow = kr + (lane & 7) + (((lane >> 3) & 1) << 3);
                ldsm_x2_trans(bb0, bb1, I + brow * ldi + nt * 8);
                mma_bf16(acc[i], a, bb0, bb1);
            }
        }
    }
    // partial: rows co = mt * 16 + g (+ 8), columns ci = nt * 8 + 2 tig (+ 1)
    const int g = lane >> 2, tig = lane & 3;
    float* dst = part + ((long long)split * 27 + t) * Cout * Cin;
#pragma unroll
    for (int i = 0; i < kWgTiles; ++i) {
        const int tile = warp + 8 * i;
        if (tile >= tiles) break;
        const int mt = tile % mt_n, nt = tile / mt_n;
        const int co = mt * 16 + g, ci = nt * 8 + 2 * tig;
        dst[co * Cin + ci] = acc[i][0];
        dst[co * Cin + ci + 1] = acc[i][1];
        dst[(co + 8) * Cin + ci] = acc[i][2];
        dst[(co + 8) * Cin + ci + 1] = acc[i][3];
    }
}

// grad[t][co][ci < cin_real] = sum over splits (fixed order)
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, int nsplit, int Cout, int Cin, int cin_real,
                                    float* __restrict__ grad) {
    const long long n = 27LL * Cout * cin_real;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(i % cin_real);
        const long long tco = i / cin_real;
        float s = 0.0f;
        for (int k = 0; k < nsplit; ++k) s += part[((long long)k * 27 * Cout + tco) * Cin + ci];
        grad[i] = s;
    }
}

// ---------------------------------------------------------------------------
// elementwise kernels (channels-last; ld = row stride in elements)
// ---------------------------------------------------------------------------
#define GLOOP(i, n) \
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

// x FP32 [cin][V] -> BF16 [V][16] (channels cin .. 15 zero)
__global__ void pack_input_kernel(const float* __restrict__ x, int cin, long long V, bf16* __restrict__ out) {
    GLOOP(i, V * 16) {
        const long long vox = i >> 4;
        const int c = (int)(i & 15);
        out[i] = __float2bfloat16_rn(c < cin ? x[(long long)c * V + vox] : 0.0f);
    }
}

// 2x2x2 mean of C channels: fine [Vf][ld_in] -> coarse [Vc][C]
__global__ void pool_kernel(const bf16* __restrict__ in, int ld_in, int C, Vol vf, bf16* __restrict__ out) {
    const Vol vc{vf.D / 2, vf.H / 2, vf.W / 2};
    GLOOP(i, vc.n() * C) {
        const int c = (int)(i % C);
        const long long p = i / C;
        const int x = (int)(p % vc.W), y = (int)((p / vc.W) % vc.H), z = (int)(p / ((long long)vc.W * vc.H));
        float s = 0.0f;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int d = 0; d < 2; ++d)
                    s += __bfloat162float(in[(((long long)(2 * z + a) * vf.H + 2 * y + b) * vf.W + 2 * x + d) * ld_in + c]);
        out[i] = __float2bfloat16_rn(0.125f * s);
    }
}

// nearest upsampling: coarse [Vc][C] -> fine slice [Vf][ld_out] (channels 0 .. C)
__global__ void upsample_kernel(const bf16* __restrict__ in, int C, Vol vf, bf16* __restrict__ out, int ld_out) {
    const Vol vc{vf.D / 2, vf.H / 2, vf.W / 2};
    GLOOP(i, vf.n() * C) {
        const int c = (int)(i % C);
        const long long p = i / C;
        const int x = (int)(p % vf.W), y = (int)((p / vf.W) % vf.H), z = (int)(p / ((long long)vf.W * vf.H));
        out[p * ld_out + c] = in[(((long long)(z / 2) * vc.H + y / 2) * vc.W + x / 2) * C + c];
    }
}

// gradient of the upsampling: fine FP32 slice [Vf][ld] -> coarse FP32 [Vc][C] (sum of the 8 children)
__global__ void upsample_bwd_kernel(const float* __restrict__ g, int ld, int C, Vol vf, float* __restrict__ out) {
    const Vol vc{vf.D / 2, vf.H / 2, vf.W / 2};
    GLOOP(i, vc.n() * C) {
        const int c = (int)(i % C);
        const long long p = i / C;
        const int x = (int)(p % vc.W), y = (int)((p / vc.W) % vc.H), z = (int)(p / ((long long)vc.W * vc.H));
        float s = 0.0f;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int d = 0; d < 2; ++d) s += g[(((long long)(2 * z + a) * vf.H + 2 * y + b) * vf.W + 2 * x + d) * ld + c];
        out[i] = s;
    }
}

// gradient of the pooling, added: fine FP32 [Vf][C] += coarse FP32 [Vc][ld_c] / 8
__global__ void pool_bwd_add_kernel(const float* __restrict__ gc, int ld_c, int C, Vol vf, float* __restrict__ gf) {
    const Vol vc{vf.D / 2, vf.H / 2, vf.W / 2};
    GLOOP(i, vf.n() * C) {
        const int c = (int)(i % C);
        const long long p = i / C;
        const int x = (int)(p % vf.W), y = (int)((p / vf.W) % vf.H), z = (int)(p / ((long long)vf.W * vf.H));
        gf[i] += 0.125f * gc[(((long long)(z / 2) * vc.H + y / 2) * vc.W + x / 2) * ld_c + c];
    }
}

// copy a FP32 channel slice [V][ld] (C channels) into a dense [V][C]
__global__ void slice_copy_kernel(const float* __restrict__ g, int ld, int C, long long V, float* __restrict__ out) {
    GLOOP(i, V * C) out[i] = g[(i / C) * ld + (i % C)];
}

// signal of a ReLU layer: s = bf16(g * (act > 0)); g FP32 [V][ld_g], act BF16 [V][ld_a], s BF16 [V][C]
__global__ void mask_round_kernel(const float* __restrict__ g, int ld_g, const bf16* __restrict__ act, int ld_a, int C,
                                  long long V, bf16* __restrict__ s) {
    GLOOP(i, V * C) {
        const long long p = i / C;
        const int c = (int)(i % C);
        const float a = __bfloat162float(act[p * ld_a + c]);
        s[i] = __float2bfloat16_rn(a > 0.0f ? g[p * ld_g + c] : 0.0f);
    }
}

// 1x1 output layer: y[o][v] = b[o] + sum_c W[o][c] d[v][c] (FP32 out, channels first)
__global__ void out_fwd_kernel(const bf16* __restrict__ d, const bf16* __restrict__ W, const float* __restrict__ b,
                               int cout, long long V, float* __restrict__ y) {
    GLOOP(p, V) {
        float in[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) in[c] = __bfloat162float(d[p * 16 + c]);
        for (int o = 0; o < cout; ++o) {
            float s = b[o];
#pragma unroll
            for (int c = 0; c < 16; ++c) s = fmaf(__bfloat162float(W[o * 16 + c]), in[c], s);
            y[(long long)o * V + p] = s;
        }
    }
}

// its input gradient, masked and rounded: s[v][c] = bf16((d > 0) sum_o W[o][c] gy[o][v])
__global__ void out_bwd_kernel(const float* __restrict__ gy, const bf16* __restrict__ W, const bf16* __restrict__ d,
                               int cout, long long V, bf16* __restrict__ s) {
    GLOOP(i, V * 16) {
        const long long p = i >> 4;
        const int c = (int)(i & 15);
        float acc = 0.0f;
        for (int o = 0; o < cout; ++o) acc = fmaf(__bfloat162float(W[o * 16 + c]), gy[(long long)o * V + p], acc);
        s[i] = __float2bfloat16_rn(__bfloat162float(d[i]) > 0.0f ? acc : 0.0f);
    }
}

__device__ __forceinline__ float block_sum_f(float v) {
    __shared__ float sh[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x >> 5)) ? sh[lane] : 0.0f;
    if (wid == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// per-CTA partial sums over voxels of channel blockIdx.y; the second stage sums them in order
__global__ void chan_sum_bf16_kernel(const bf16* __restrict__ s, int C, long long V, float* __restrict__ part) {
    const int c = blockIdx.y;
    float a = 0.0f;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < V; p += (long long)gridDim.x * blockDim.x)
        a += __bfloat162float(s[p * C + c]);
    a = block_sum_f(a);
    if (threadIdx.x == 0) part[c * gridDim.x + blockIdx.x] = a;
}

// output layer: dW[o][c] = sum_v gy[o][v] d[v][c] and db[o] = sum_v gy[o][v], partials per CTA
__global__ void out_wgrad_kernel(const float* __restrict__ gy, const bf16* __restrict__ d, int cout, long long V,
                                 float* __restrict__ part) {
    const int k = blockIdx.y;              // k = o * 17 + c, c = 16 for the bias
    const int o = k / 17, c = k % 17;
    float a = 0.0f;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < V; p += (long long)gridDim.x * blockDim.x)
        a = fmaf(gy[(long long)o * V + p], c < 16 ? __bfloat162float(d[p * 16 + c]) : 1.0f, a);
    a = block_sum_f(a);
    if (threadIdx.x == 0) part[k * gridDim.x + blockIdx.x] = a;
}

__global__ void part_reduce_kernel(const float* __restrict__ part, int nparts, int n, float* __restrict__ out,
                                   const int* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.0f;
    for (int k = 0; k < nparts; ++k) s += part[i * nparts + k];
    out[dst ? dst[i] : i] = s;
}

// MSE: g = 2 (y - t) / N; per-CTA partial sums of (y - t)^2
__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t, long long n,
                           float* __restrict__ g, float* __restrict__ part) {
    float s = 0.0f;
    const float scale = 2.0f / (float)n;
    GLOOP(i, n) {
        const float d = y[i] - t[i];
        g[i] = scale * d;
        s = fmaf(d, d, s);
    }
    s = block_sum_f(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void adam_kernel(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ vv,
                            const float* __restrict__ g, int n, float lr, float b1, float b2, float c1, float c2,
                            float eps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * vv[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    vv[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// BF16 weights of a layer: wf[t][co][ci_pad] (forward) and the transpose wb[t][ci_pad][co]
// (data gradient, which reads the neighbour at -d_t); channels ci >= cin_real are zero
__global__ void prep_weights_kernel(const float* __restrict__ theta, int taps, int cout, int cin_real, int cin_pad,
                                    bf16* __restrict__ wf, bf16* __restrict__ wb) {
    const int n = taps * cout * cin_pad;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int ci = i % cin_pad, co = (i / cin_pad) % cout, t = i / (cin_pad * cout);
    const float w = ci < cin_real ? theta[((long long)t * cout + co) * cin_real + ci] : 0.0f;
    const bf16 r = __float2bfloat16_rn(w);
    wf[i] = r;
    if (wb) wb[((long long)t * cin_pad + ci) * cout + co] = r;
}

struct LayerDef {
    int cin, cout, taps, cin_pad;
    long long woff, boff;        // offsets in theta
    long long wf, wb;            // offsets in the BF16 weight buffers
};

}  // namespace

struct ht_unet {
    int cin = 8, cout = 2, device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int np = 0;
    LayerDef L[kLayers];
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    bf16 *wf = nullptr, *wb = nullptr;
    long long nwf = 0;
    // activations (BF16 channels-last) and gradients, sized for the largest grid seen
    long long cap = 0;
    bf16 *xin = nullptr, *a0 = nullptr, *cat1 = nullptr, *p1 = nullptr, *a2 = nullptr, *cat2 = nullptr;
    bf16 *p2 = nullptr, *a4 = nullptr, *cat3 = nullptr, *p3 = nullptr, *a6 = nullptr, *a7 = nullptr;
    bf16 *d3a = nullptr, *d3 = nullptr, *d2a = nullptr, *d2 = nullptr, *d1a = nullptr, *d1 = nullptr, *sig = nullptr;
    float *y = nullptr, *gy = nullptr, *gin = nullptr, *gup = nullptr, *ge1 = nullptr, *ge2 = nullptr, *ge3 = nullptr;
    float *wpart = nullptr, *cpart = nullptr;
    int* bidx = nullptr;
    int step = 0;
    bool weights_ready = false;
    std::string err;
};

namespace {

int ufail(ht_unet* u, int code, const char* msg) {
    if (u) u->err = msg;
    return code;
}

int grid_for(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b > 8192 ? 8192 : (b < 1 ? 1 : b));
}

void build_layers(ht_unet* u) {
    const int c1 = kW1, c2 = kW2, c3 = kW3, c4 = kW4;
    const int def[kLayers][3] = {{u->cin, c1, 27}, {c1, c1, 27}, {c1, c2, 27}, {c2, c2, 27}, {c2, c3, 27},
                                 {c3, c3, 27},     {c3, c4, 27}, {c4, c4, 27}, {c4 + c3, c3, 27}, {c3, c3, 27},
                                 {c3 + c2, c2, 27}, {c2, c2, 27}, {c2 + c1, c1, 27}, {c1, c1, 27}, {c1, u->cout, 1}};
    long long o = 0, w = 0;
    for (int l = 0; l < kLayers; ++l) {
        LayerDef& d = u->L[l];
        d.cin = def[l][0];
        d.cout = def[l][1];
        d.taps = def[l][2];
        d.cin_pad = l == 0 ? 16 : d.cin;
        d.woff = o;
        o += (long long)d.taps * d.cout * d.cin;
        d.boff = o;
        o += d.cout;
        d.wf = w;
        d.wb = w + (long long)d.taps * d.cout * d.cin_pad;
        w += 2LL * d.taps * d.cout * d.cin_pad;
    }
    u->np = (int)o;
    u->nwf = w;
}

template <typename T>
int alloc(ht_unet* u, T** p, long long n) {
    if (*p) cudaFree(*p);
    *p = nullptr;
    if (n <= 0) n = 1;
    if (cudaMalloc(p, (size_t)n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return ufail(u, HT_ENOMEM, "U-Net buffers do not fit in device memory");
    }
    return HT_OK;
}

int ensure(ht_unet* u, const Vol& v) {
    const long long V0 = v.n();
    if (V0 <= u->cap) return HT_OK;
    const long long V1 = V0 / 8, V2 = V0 / 64, V3 = V0 / 512;
    int rc = HT_OK;
    struct B { bf16** p; long long n; } bb[] = {
        {&u->xin, V0 * 16}, {&u->a0, V0 * 16}, {&u->cat1, V0 * 48}, {&u->p1, V1 * 16}, {&u->a2, V1 * 32},
        {&u->cat2, V1 * 80}, {&u->p2, V2 * 32}, {&u->a4, V2 * 48}, {&u->cat3, V2 * 112}, {&u->p3, V3 * 48},
        {&u->a6, V3 * 64}, {&u->a7, V3 * 64}, {&u->d3a, V2 * 48}, {&u->d3, V2 * 48}, {&u->d2a, V1 * 32},
        {&u->d2, V1 * 32}, {&u->d1a, V0 * 16}, {&u->d1, V0 * 16}, {&u->sig, V0 * 16}};
    for (auto& b : bb)
        if (rc == HT_OK) rc = alloc(u, b.p, b.n);
    struct F { float** p; long long n; } ff[] = {
        {&u->y, 2 * V0}, {&u->gy, 2 * V0}, {&u->gin, V0 * 48}, {&u->gup, V1 * 32}, {&u->ge1, V0 * 16},
        {&u->ge2, V1 * 32}, {&u->ge3, V2 * 48}};
    for (auto& f : ff)
        if (rc == HT_OK) rc = alloc(u, f.p, f.n);
    if (rc == HT_OK) u->cap = V0;
    return rc;
}

size_t conv_smem(int NT) { return (size_t)27 * NT * 8 * 24 * sizeof(bf16); }

template <int NT>
void launch_conv_nt(ht_unet* u, const bf16* in, int ld_in, int K, const bf16* W, int Nout, int n0, const float* bias,
                    bf16* ob, float* of, int ld_out, int relu, const Vol& v, int flip) {
    const size_t smem = conv_smem(NT);
    cudaFuncSetAttribute(conv3_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const long long blocks = (v.n() + kConvVox - 1) / kConvVox;
    conv3_kernel<NT><<<(unsigned)blocks, kThreads, smem, u->stream>>>(in, ld_in, K, W, Nout, n0, bias, ob, of, ld_out,
                                                                      relu, v, flip);
}

// all Nout output channels, in passes of at most 64
void conv(ht_unet* u, const bf16* in, int ld_in, int K, const bf16* W, int Nout, const float* bias, bf16* ob,
          float* of, int ld_out, int relu, const Vol& v, int flip) {
    const int passes = (Nout + 63) / 64;
    const int per = Nout / passes;          // 112 -> 2 x 56, 80 -> 2 x 40, others one pass
    for (int k = 0; k < passes; ++k) {
        const int n0 = k * per;
        switch (per / 8) {
            case 2: launch_conv_nt<2>(u, in, ld_in, K, W, Nout, n0, bias, ob, of, ld_out, relu, v, flip); break;
            case 4: launch_conv_nt<4>(u, in, ld_in, K, W, Nout, n0, bias, ob, of, ld_out, relu, v, flip); break;
            case 5: launch_conv_nt<5>(u, in, ld_in, K, W, Nout, n0, bias, ob, of, ld_out, relu, v, flip); break;
            case 6: launch_conv_nt<6>(u, in, ld_in, K, W, Nout, n0, bias, ob, of, ld_out, relu, v, flip); break;
            case 7: launch_conv_nt<7>(u, in, ld_in, K, W, Nout, n0, bias, ob, of, ld_out, relu, v, flip); break;
            default: launch_conv_nt<8>(u, in, ld_in, K, W, Nout, n0, bias, ob, of, ld_out, relu, v, flip); break;
        }
    }
}

void conv_fwd(ht_unet* u, int l, const bf16* in, int ld_in, bf16* out, int ld_out, const Vol& v) {
    const LayerDef& d = u->L[l];
    conv(u, in, ld_in, d.cin_pad, u->wf + d.wf, d.cout, u->theta + d.boff, out, nullptr, ld_out, 1, v, 0);
}

// data gradient of layer l: gin [V][cin] (FP32) from its signal [V][cout]
void conv_dgrad(ht_unet* u, int l, const bf16* sig, const Vol& v) {
    const LayerDef& d = u->L[l];
    conv(u, sig, d.cout, d.cout, u->wf + d.wb, d.cin_pad, nullptr, nullptr, u->gin, d.cin_pad, 0, v, 1);
}

// weight and bias gradients of layer l from its input slice and its signal
void conv_wgrad(ht_unet* u, int l, const bf16* in, int ld_in, const bf16* sig, const Vol& v) {
    const LayerDef& d = u->L[l];
    const long long V = v.n();
    const long long nblk = (V + kWgVox - 1) / kWgVox;
    const int nsplit = (int)(nblk < kWgSplit ? nblk : kWgSplit);
    const size_t smem = (size_t)kWgVox * ((d.cout + 8) + (d.cin_pad + 8)) * sizeof(bf16);
    cudaFuncSetAttribute(wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    wgrad_kernel<<<dim3(nsplit, 27), kThreads, smem, u->stream>>>(sig, d.cout, in, ld_in, d.cin_pad, v, u->wpart,
                                                                   nsplit);
    const long long n = 27LL * d.cout * d.cin;
    wgrad_reduce_kernel<<<grid_for(n), 256, 0, u->stream>>>(u->wpart, nsplit, d.cout, d.cin_pad, d.cin,
                                                             u->grad + d.woff);
    const int nb = 64;
    chan_sum_bf16_kernel<<<dim3(nb, d.cout), 256, 0, u->stream>>>(sig, d.cout, V, u->cpart);
    part_reduce_kernel<<<1, 128, 0, u->stream>>>(u->cpart, nb, d.cout, u->grad + d.boff, nullptr);
}

void prep_weights(ht_unet* u) {
    for (int l = 0; l < kLayers; ++l) {
        const LayerDef& d = u->L[l];
        const int n = d.taps * d.cout * d.cin_pad;
        prep_weights_kernel<<<(n + 255) / 256, 256, 0, u->stream>>>(u->theta + d.woff, d.taps, d.cout, d.cin,
                                                                   d.cin_pad, u->wf + d.wf,
                                                                   l > 0 && l < 14 ? u->wf + d.wb : nullptr);
    }
    u->weights_ready = true;
}

int forward(ht_unet* u, const float* x, const Vol& v0) {
    if (!u->weights_ready) prep_weights(u);
    const Vol v1{v0.D / 2, v0.H / 2, v0.W / 2}, v2{v1.D / 2, v1.H / 2, v1.W / 2}, v3{v2.D / 2, v2.H / 2, v2.W / 2};
    pack_input_kernel<<<grid_for(v0.n() * 16), 256, 0, u->stream>>>(x, u->cin, v0.n(), u->xin);
    conv_fwd(u, 0, u->xin, 16, u->a0, 16, v0);
    conv_fwd(u, 1, u->a0, 16, u->cat1 + kW2, 48, v0);                       // e1 -> cat1[:, 32:48]
    pool_kernel<<<grid_for(v1.n() * kW1), 256, 0, u->stream>>>(u->cat1 + kW2, 48, kW1, v0, u->p1);
    conv_fwd(u, 2, u->p1, 16, u->a2, 32, v1);
    conv_fwd(u, 3, u->a2, 32, u->cat2 + kW3, 80, v1);                       // e2 -> cat2[:, 48:80]
    pool_kernel<<<grid_for(v2.n() * kW2), 256, 0, u->stream>>>(u->cat2 + kW3, 80, kW2, v1, u->p2);
    conv_fwd(u, 4, u->p2, 32, u->a4, 48, v2);
    conv_fwd(u, 5, u->a4, 48, u->cat3 + kW4, 112, v2);                      // e3 -> cat3[:, 64:112]
    pool_kernel<<<grid_for(v3.n() * kW3), 256, 0, u->stream>>>(u->cat3 + kW4, 112, kW3, v2, u->p3);
    conv_fwd(u, 6, u->p3, 48, u->a6, 64, v3);
    conv_fwd(u, 7, u->a6, 64, u->a7, 64, v3);
    upsample_kernel<<<grid_for(v2.n() * kW4), 256, 0, u->stream>>>(u->a7, kW4, v2, u->cat3, 112);
    conv_fwd(u, 8, u->cat3, 112, u->d3a, 48, v2);
    conv_fwd(u, 9, u->d3a, 48, u->d3, 48, v2);
    upsample_kernel<<<grid_for(v1.n() * kW3), 256, 0, u->stream>>>(u->d3, kW3, v1, u->cat2, 80);
    conv_fwd(u, 10, u->cat2, 80, u->d2a, 32, v1);
    conv_fwd(u, 11, u->d2a, 32, u->d2, 32, v1);
    upsample_kernel<<<grid_for(v0.n() * kW2), 256, 0, u->stream>>>(u->d2, kW2, v0, u->cat1, 48);
    conv_fwd(u, 12, u->cat1, 48, u->d1a, 16, v0);
    conv_fwd(u, 13, u->d1a, 16, u->d1, 16, v0);
    const LayerDef& o = u->L[14];
    out_fwd_kernel<<<grid_for(v0.n()), 256, 0, u->stream>>>(u->d1, u->wf + o.wf, u->theta + o.boff, u->cout, v0.n(), u->y);
    return cudaGetLastError() == cudaSuccess ? HT_OK : ufail(u, HT_ECUDA, "forward launch failed");
}

// the signal of layer l (output act, FP32 gradient g [V][ld_g]) into u->sig
void signal(ht_unet* u, const float* g, int ld_g, const bf16* act, int ld_a, int C, const Vol& v) {
    mask_round_kernel<<<grid_for(v.n() * C), 256, 0, u->stream>>>(g, ld_g, act, ld_a, C, v.n(), u->sig);
}

int backward(ht_unet* u, const float* target, const Vol& v0, double* loss) {
    const Vol v1{v0.D / 2, v0.H / 2, v0.W / 2}, v2{v1.D / 2, v1.H / 2, v1.W / 2}, v3{v2.D / 2, v2.H / 2, v2.W / 2};
    const long long ny = (long long)u->cout * v0.n();
    const int G = grid_for(ny) > 1024 ? 1024 : grid_for(ny);
    mse_kernel<<<G, 256, 0, u->stream>>>(u->y, target, ny, u->gy, u->cpart + 4096);
    // output layer (1x1, FP32 signal)
    {
        const LayerDef& o = u->L[14];
        const int nb = 64;
        out_wgrad_kernel<<<dim3(nb, u->cout * 17), 256, 0, u->stream>>>(u->gy, u->d1, u->cout, v0.n(), u->cpart);
        part_reduce_kernel<<<1, 64, 0, u->stream>>>(u->cpart, nb, u->cout * 17, u->grad, u->bidx);
        (void)o;
        out_bwd_kernel<<<grid_for(v0.n() * 16), 256, 0, u->stream>>>(u->gy, u->wf + o.wf, u->d1, u->cout, v0.n(), u->sig);
    }
    // level 1 decoder
    conv_wgrad(u, 13, u->d1a, 16, u->sig, v0);
    conv_dgrad(u, 13, u->sig, v0);
    signal(u, u->gin, 16, u->d1a, 16, 16, v0);
    conv_wgrad(u, 12, u->cat1, 48, u->sig, v0);
    conv_dgrad(u, 12, u->sig, v0);                                     // gin [V0][48]: up d2 | e1
    slice_copy_kernel<<<grid_for(v0.n() * kW1), 256, 0, u->stream>>>(u->gin + kW2, 48, kW1, v0.n(), u->ge1);
    upsample_bwd_kernel<<<grid_for(v1.n() * kW2), 256, 0, u->stream>>>(u->gin, 48, kW2, v0, u->gup);
    // level 2 decoder
    signal(u, u->gup, kW2, u->d2, 32, 32, v1);
    conv_wgrad(u, 11, u->d2a, 32, u->sig, v1);
    conv_dgrad(u, 11, u->sig, v1);
    signal(u, u->gin, 32, u->d2a, 32, 32, v1);
    conv_wgrad(u, 10, u->cat2, 80, u->sig, v1);
    conv_dgrad(u, 10, u->sig, v1);                                     // gin [V1][80]: up d3 | e2
    slice_copy_kernel<<<grid_for(v1.n() * kW2), 256, 0, u->stream>>>(u->gin + kW3, 80, kW2, v1.n(), u->ge2);
    upsample_bwd_kernel<<<grid_for(v2.n() * kW3), 256, 0, u->stream>>>(u->gin, 80, kW3, v1, u->gup);
    // level 3 decoder
    signal(u, u->gup, kW3, u->d3, 48, 48, v2);
    conv_wgrad(u, 9, u->d3a, 48, u->sig, v2);
    conv_dgrad(u, 9, u->sig, v2);
    signal(u, u->gin, 48, u->d3a, 48, 48, v2);
    conv_wgrad(u, 8, u->cat3, 112, u->sig, v2);
    conv_dgrad(u, 8, u->sig, v2);                                      // gin [V2][112]: up a7 | e3
    slice_copy_kernel<<<grid_for(v2.n() * kW3), 256, 0, u->stream>>>(u->gin + kW4, 112, kW3, v2.n(), u->ge3);
    upsample_bwd_kernel<<<grid_for(v3.n() * kW4), 256, 0, u->stream>>>(u->gin, 112, kW4, v2, u->gup);
    // level 4
    signal(u, u->gup, kW4, u->a7, 64, 64, v3);
    conv_wgrad(u, 7, u->a6, 64, u->sig, v3);
    conv_dgrad(u, 7, u->sig, v3);
    signal(u, u->gin, 64, u->a6, 64, 64, v3);
    conv_wgrad(u, 6, u->p3, 48, u->sig, v3);
    conv_dgrad(u, 6, u->sig, v3);                                      // gin [V3][48] -> e3
    pool_bwd_add_kernel<<<grid_for(v2.n() * kW3), 256, 0, u->stream>>>(u->gin, 48, kW3, v2, u->ge3);
    // level 3 encoder
    signal(u, u->ge3, kW3, u->cat3 + kW4, 112, 48, v2);
    conv_wgrad(u, 5, u->a4, 48, u->sig, v2);
    conv_dgrad(u, 5, u->sig, v2);
    signal(u, u->gin, 48, u->a4, 48, 48, v2);
    conv_wgrad(u, 4, u->p2, 32, u->sig, v2);
    conv_dgrad(u, 4, u->sig, v2);                                      // gin [V2][32] -> e2
    pool_bwd_add_kernel<<<grid_for(v1.n() * kW2), 256, 0, u->stream>>>(u->gin, 32, kW2, v1, u->ge2);
    // level 2 encoder
    signal(u, u->ge2, kW2, u->cat2 + kW3, 80, 32, v1);
    conv_wgrad(u, 3, u->a2, 32, u->sig, v1);
    conv_dgrad(u, 3, u->sig, v1);
    signal(u, u->gin, 32, u->a2, 32, 32, v1);
    conv_wgrad(u, 2, u->p1, 16, u->sig, v1);
    conv_dgrad(u, 2, u->sig, v1);                                      // gin [V1][16] -> e1
    pool_bwd_add_kernel<<<grid_for(v0.n() * kW1), 256, 0, u->stream>>>(u->gin, 16, kW1, v0, u->ge1);
    // level 1 encoder
    signal(u, u->ge1, kW1, u->cat1 + kW2, 48, 16, v0);
    conv_wgrad(u, 1, u->a0, 16, u->sig, v0);
    conv_dgrad(u, 1, u->sig, v0);
    signal(u, u->gin, 16, u->a0, 16, 16, v0);
    conv_wgrad(u, 0, u->xin, 16, u->sig, v0);
    if (cudaGetLastError() != cudaSuccess) return ufail(u, HT_ECUDA, "backward launch failed");
    if (loss) {
        std::vector<float> h(G);
        if (cudaMemcpyAsync(h.data(), u->cpart + 4096, G * sizeof(float), cudaMemcpyDeviceToHost, u->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(u->stream) != cudaSuccess)
            return ufail(u, HT_ECUDA, "loss readback failed");
        double s = 0;
        for (float f : h) s += f;
        *loss = s / (double)ny;
    }
    return HT_OK;
}

bool dims_ok(int D, int H, int W) { return D >= 8 && H >= 8 && W >= 8 && D % 8 == 0 && H % 8 == 0 && W % 8 == 0; }

}  // namespace

cudaStream_t ht_unet_stream_internal(ht_unet* u) { return u ? u->stream : nullptr; }

extern "C" {

int ht_unet_create(ht_unet** out, int cin, int cout, int device, void* stream) {
    if (!out || cin < 1 || cin > 16 || cout != 2) return HT_EINVAL;
    *out = nullptr;
    ht_unet* u = new ht_unet();
    u->cin = cin;
    u->cout = cout;
    u->device = device;
    if (cudaSetDevice(device) != cudaSuccess) { delete u; return HT_ECUDA; }
    if (stream) u->stream = (cudaStream_t)stream;
    else { cudaStreamCreateWithFlags(&u->stream, cudaStreamNonBlocking); u->own_stream = true; }
    build_layers(u);
    const int o = u->np;
    // gradient positions of the output layer's weights and biases (o * 17 + c order)
    std::vector<int> bidx(cout * 17);
    for (int oo = 0; oo < cout; ++oo)
        for (int c = 0; c < 17; ++c)
            bidx[oo * 17 + c] = c < 16 ? (int)(u->L[14].woff + oo * 16 + c) : (int)(u->L[14].boff + oo);
    int largest_part = 0;
    for (int l = 0; l < kLayers; ++l) {
        const int s = kWgSplit * 27 * u->L[l].cout * u->L[l].cin_pad;
        if (s > largest_part) largest_part = s;
    }
    if (alloc(u, &u->theta, o) || alloc(u, &u->m, o) || alloc(u, &u->v, o) || alloc(u, &u->grad, o) ||
        alloc(u, &u->wf, u->nwf) || alloc(u, &u->wpart, largest_part) || alloc(u, &u->cpart, 8192) ||
        alloc(u, &u->bidx, cout * 17)) {
        ht_unet_destroy(u);
        return HT_ENOMEM;
    }
    cudaMemcpyAsync(u->bidx, bidx.data(), bidx.size() * sizeof(int), cudaMemcpyHostToDevice, u->stream);
    cudaMemsetAsync(u->theta, 0, o * sizeof(float), u->stream);
    cudaMemsetAsync(u->m, 0, o * sizeof(float), u->stream);
    cudaMemsetAsync(u->v, 0, o * sizeof(float), u->stream);
    cudaMemsetAsync(u->grad, 0, o * sizeof(float), u->stream);
    if (cudaStreamSynchronize(u->stream) != cudaSuccess) { ht_unet_destroy(u); return HT_ECUDA; }
    *out = u;
    return HT_OK;
}

void ht_unet_destroy(ht_unet* u) {
    if (!u) return;
    cudaSetDevice(u->device);
    if (u->stream) cudaStreamSynchronize(u->stream);
    void* bufs[] = {u->theta, u->m, u->v, u->grad, u->wf, u->wpart, u->cpart, u->bidx, u->xin, u->a0, u->cat1,
                    u->p1, u->a2, u->cat2, u->p2, u->a4, u->cat3, u->p3, u->a6, u->a7, u->d3a, u->d3, u->d2a,
                    u->d2, u->d1a, u->d1, u->sig, u->y, u->gy, u->gin, u->gup, u->ge1, u->ge2, u->ge3};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (u->own_stream && u->stream) cudaStreamDestroy(u->stream);
    delete u;
}

int ht_unet_num_params(const ht_unet* u) { return u ? u->np : 0; }

const char* ht_unet_last_error(const ht_unet* u) { return u ? u->err.c_str() : ""; }

int ht_unet_set_params(ht_unet* u, const float* theta) {
    if (!u || !theta) return HT_EINVAL;
    cudaSetDevice(u->device);
    if (cudaMemcpyAsync(u->theta, theta, u->np * sizeof(float), cudaMemcpyHostToDevice, u->stream) != cudaSuccess)
        return ufail(u, HT_ECUDA, "parameter upload failed");
    cudaMemsetAsync(u->m, 0, u->np * sizeof(float), u->stream);
    cudaMemsetAsync(u->v, 0, u->np * sizeof(float), u->stream);
    u->step = 0;
    prep_weights(u);
    return cudaStreamSynchronize(u->stream) == cudaSuccess ? HT_OK : ufail(u, HT_ECUDA, "sync failed");
}

int ht_unet_get_params(ht_unet* u, float* theta) {
    if (!u || !theta) return HT_EINVAL;
    cudaSetDevice(u->device);
    if (cudaMemcpyAsync(theta, u->theta, u->np * sizeof(float), cudaMemcpyDeviceToHost, u->stream) != cudaSuccess ||
        cudaStreamSynchronize(u->stream) != cudaSuccess)
        return ufail(u, HT_ECUDA, "parameter readback failed");
    return HT_OK;
}

int ht_unet_forward(ht_unet* u, const float* x, int D, int H, int W, float* y) {
    if (!u || !x || !y) return HT_EINVAL;
    if (!dims_ok(D, H, W)) return ufail(u, HT_EINVAL, "grid sizes must be multiples of 8");
    cudaSetDevice(u->device);
    const Vol v{D, H, W};
    int rc = ensure(u, v);
    if (rc != HT_OK) return rc;
    rc = forward(u, x, v);
    if (rc != HT_OK) return rc;
    if (cudaMemcpyAsync(y, u->y, (size_t)u->cout * v.n() * sizeof(float), cudaMemcpyDeviceToDevice, u->stream) !=
        cudaSuccess)
        return ufail(u, HT_ECUDA, "output copy failed");
    return HT_OK;
}

int ht_unet_loss_grad(ht_unet* u, const float* x, const float* target, int D, int H, int W, double* loss,
                      float* grad_host) {
    if (!u || !x || !target) return HT_EINVAL;
    if (!dims_ok(D, H, W)) return ufail(u, HT_EINVAL, "grid sizes must be multiples of 8");
    cudaSetDevice(u->device);
    const Vol v{D, H, W};
    int rc = ensure(u, v);
    if (rc == HT_OK) rc = forward(u, x, v);
    if (rc == HT_OK) rc = backward(u, target, v, loss);
    if (rc == HT_OK && grad_host) {
        if (cudaMemcpyAsync(grad_host, u->grad, u->np * sizeof(float), cudaMemcpyDeviceToHost, u->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(u->stream) != cudaSuccess)
            return ufail(u, HT_ECUDA, "gradient readback failed");
    }
    return rc;
}

int ht_unet_train_step(ht_unet* u, const float* x, const float* target, int D, int H, int W, float lr,
                       double* loss) {
    if (!u || !x || !target || !(lr > 0)) return HT_EINVAL;
    int rc = ht_unet_loss_grad(u, x, target, D, H, W, loss, nullptr);
    if (rc != HT_OK) return rc;
    u->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)u->step), c2 = 1.f - powf(b2, (float)u->step);
    adam_kernel<<<(u->np + 255) / 256, 256, 0, u->stream>>>(u->theta, u->m, u->v, u->grad, u->np, lr, b1, b2, c1, c2,
                                                            1e-8f);
    prep_weights(u);
    return cudaGetLastError() == cudaSuccess ? HT_OK : ufail(u, HT_ECUDA, "adam launch failed");
}

}  // extern "C"
