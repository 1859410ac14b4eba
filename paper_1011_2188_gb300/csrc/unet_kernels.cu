// Kernels of the learned denoiser (3-D U-Net over dose grids): BF16
// tensor-core convolutions as implicit GEMMs with FP32 accumulation, their
// data and weight gradients, and the element-wise pieces of the network and
// its training (ReLU gradient, nearest upsampling, channel concatenation,
// mean-squared error, Adam).  Activations are channels-last,
// [batch][d][h][w][c] in BF16; weights [c_out][k^3][c_in].
//
// conv_igemm_kernel computes out[r][n] = sum_k A[r][k] * B[n][k] with
//   forward: r = output voxel, n = output channel, k = (tap, input channel),
//            A gathered from the input at voxel r * stride - pad + tap;
//   data gradient: r = input voxel, n = input channel, k = (tap, output
//            channel), A gathered from the output gradient at
//            (r + pad - tap) / stride when that divides exactly.
// Tiles: 128 rows x NT columns per CTA of four warps, K in steps of 16 channels
// of one tap, operands staged through shared memory with cp.async (zero fill
// for padding), mma.sync m16n8k16 BF16 -> FP32.  It serves the 2^3 stride-2
// and 1^3 layers; the 3^3 stride-1 layers (nearly all of the network's FLOPs)
// run on the tcgen05 tensor cores with TMEM accumulators (conv3_tc_kernel,
// persistent and pipelined).

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "fdc_internal.h"
#include "unet_internal.h"

namespace fdc {
namespace {

constexpr int kRows = 128;       // rows (voxels) per CTA
constexpr int kRowBytes = 48;    // 16 BF16 (32 B) padded to 48 B: conflict-free fragment loads

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(n));
}
// The same with L1 allocation: for data that many CTAs on an SM read (weights).
__device__ __forceinline__ void cp_async16_ca(void *smem, const void *gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N)); }

__device__ __forceinline__ void mma_bf16(float c[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned lds32(const unsigned char *p) { return *(const unsigned *)p; }

struct RowCoord {
    int b, d, h, w;
    bool valid;
};

__device__ __forceinline__ RowCoord row_coord(long long r, long long rows, int D, int H, int W) {
    RowCoord c;
    c.valid = r < rows;
    if (!c.valid) r = 0;
    c.w = (int)(r % W);
    long long q = r / W;
    c.h = (int)(q % H);
    q /= H;
    c.d = (int)(q % D);
    c.b = (int)(q / D);
    return c;
}

// Source voxel of row c for tap (kd, kh, kw); -1 when outside (padding).
template <int MODE>
__device__ __forceinline__ long long src_voxel(const RowCoord &c, int kd, int kh, int kw, const Conv3dArgs &g) {
    int sd, sh, sw, Ds, Hs, Ws;
    if (MODE == 0) {
        Ds = g.in_d; Hs = g.in_h; Ws = g.in_w;
        sd = c.d * g.stride - g.pad + kd;
        sh = c.h * g.stride - g.pad + kh;
        sw = c.w * g.stride - g.pad + kw;
    } else {
        Ds = g.out_d; Hs = g.out_h; Ws = g.out_w;
        int td = c.d + g.pad - kd, th = c.h + g.pad - kh, tw = c.w + g.pad - kw;
        if (td < 0 || th < 0 || tw < 0 || td % g.stride || th % g.stride || tw % g.stride) return -1;
        sd = td / g.stride; sh = th / g.stride; sw = tw / g.stride;
    }
    if (!c.valid || sd < 0 || sh < 0 || sw < 0 || sd >= Ds || sh >= Hs || sw >= Ws) return -1;
    return (((long long)c.b * Ds + sd) * Hs + sh) * (long long)Ws + sw;
}

template <int MODE, int NT>
__global__ void __launch_bounds__(128) conv_igemm_kernel(const Conv3dArgs g, const __nv_bfloat16 *src,
                                                         const __nv_bfloat16 *wt, const float *bias,
                                                         __nv_bfloat16 *out_bf16, float *out_f32) {
    __shared__ __align__(16) unsigned char sA[2][kRows * kRowBytes];
    __shared__ __align__(16) unsigned char sB[2][NT * kRowBytes];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int grp = lane >> 2, tig = lane & 3;
    // row space and source channels per mode
    const int Dr = MODE == 0 ? g.out_d : g.in_d, Hr = MODE == 0 ? g.out_h : g.in_h;
    const int Wr = MODE == 0 ? g.out_w : g.in_w;
    const int Cs = MODE == 0 ? g.c_in : g.c_out;   // gathered channels (K per tap)
    const int Nn = MODE == 0 ? g.c_out : g.c_in;   // output channels
    // Data gradient of a convolution whose kernel tiles its input (stride =
    // ksize, no padding: the 2^3 stride-2 down-convolutions): input voxel
    // (d, h, w) receives exactly one tap, (d, h, w) mod stride.  The rows are
    // then the input voxels of one parity class (blockIdx.z), a sub-grid of
    // stride^3 spacing, and K runs over that one tap's channels only.
    const bool par = MODE == 1 && g.stride == g.ksize && g.pad == 0;
    int pd = 0, ph = 0, pw = 0, Dq = Dr, Hq = Hr, Wq = Wr;
    if (par) {
        const int st = g.stride, cls = blockIdx.z;
        pd = cls / (st * st); ph = (cls / st) % st; pw = cls % st;
        Dq = (Dr - pd + st - 1) / st; Hq = (Hr - ph + st - 1) / st; Wq = (Wr - pw + st - 1) / st;
    }
    const long long rows = (long long)g.batch * Dq * Hq * Wq;
    const long long r0 = (long long)blockIdx.x * kRows;
    if (r0 >= rows) return;  // parity classes with fewer rows than the grid
    const int n0 = blockIdx.y * NT;
    const int taps = g.ksize * g.ksize * g.ksize;
    const int tap_par = (pd * g.ksize + ph) * g.ksize + pw;
    const int csteps = Cs / 16;
    const int ksteps = par ? csteps : taps * csteps;
    // forward with a K split (blockIdx.z: the coarse layers, whose few row
    // tiles would leave most SMs idle): this CTA's K steps [k_lo, k_hi), its
    // FP32 partial sums stored without bias or activation to out_f32's slice z
    const int nsplit = MODE == 0 ? (int)gridDim.z : 1;
    const int k_lo = (int)((long long)ksteps * (MODE == 0 ? blockIdx.z : 0) / nsplit);
    const int k_hi = (int)((long long)ksteps * ((MODE == 0 ? blockIdx.z : 0) + 1) / nsplit);
    // the voxel (in the D x H x W row space) of row r of this grid
    auto row_voxel = [&](long long r, RowCoord &c) {
        c = row_coord(r, rows, Dq, Hq, Wq);
        if (par) {
            c.d = c.d * g.stride + pd;
            c.h = c.h * g.stride + ph;
            c.w = c.w * g.stride + pw;
        }
        return (((long long)c.b * Dr + c.d) * Hr + c.h) * (long long)Wr + c.w;
    };
    // this thread gathers row r0 + tid
    RowCoord rc;
    row_voxel(r0 + tid, rc);

    auto load_stage = [&](int buf, int ks) {
        const int tap = par ? tap_par : ks / csteps, c0 = (ks % csteps) * 16;
        const int kd = tap / (g.ksize * g.ksize), kh = (tap / g.ksize) % g.ksize, kw = tap % g.ksize;
        const long long sv = src_voxel<MODE>(rc, kd, kh, kw, g);
        const __nv_bfloat16 *p = sv >= 0 ? src + sv * Cs + c0 : src;
        unsigned char *dst = sA[buf] + tid * kRowBytes;
        cp_async16(dst, p, sv >= 0);
        cp_async16(dst + 16, p + 8, sv >= 0);
        for (int i = tid; i < NT * 2; i += 128) {
            const int n = i >> 1, half = i & 1;
            const bool ok = n0 + n < Nn;
            const __nv_bfloat16 *q = ok ? wt + ((long long)(n0 + n) * taps + tap) * Cs + c0 + half * 8 : wt;
            cp_async16(sB[buf] + n * kRowBytes + half * 16, q, ok);
        }
    };

    float acc[2][NT / 8][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < NT / 8; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;

    load_stage(0, k_lo);
    cp_async_commit();
    for (int ks = k_lo; ks < k_hi; ++ks) {
        const int buf = (ks - k_lo) & 1;
        if (ks + 1 < k_hi) load_stage(buf ^ 1, ks + 1);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const unsigned char *A = sA[buf];
        const unsigned char *B = sB[buf];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int ra = warp * 32 + mt * 16 + grp;
            const unsigned a0 = lds32(A + ra * kRowBytes + tig * 4);
            const unsigned a1 = lds32(A + (ra + 8) * kRowBytes + tig * 4);
            const unsigned a2 = lds32(A + ra * kRowBytes + 16 + tig * 4);
            const unsigned a3 = lds32(A + (ra + 8) * kRowBytes + 16 + tig * 4);
#pragma unroll
            for (int nt = 0; nt < NT / 8; ++nt) {
                const int nb = nt * 8 + grp;
                const unsigned b0 = lds32(B + nb * kRowBytes + tig * 4);
                const unsigned b1 = lds32(B + nb * kRowBytes + 16 + tig * 4);
                mma_bf16(acc[mt][nt], a0, a1, a2, a3, b0, b1);
            }
        }
        __syncthreads();
    }
    cp_async_wait<0>();
    if (nsplit > 1) out_f32 += (long long)blockIdx.z * rows * Nn;

    // epilogue: bias, ReLU, store (a split's partials: neither)
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const long long rr = r0 + warp * 32 + mt * 16 + grp + half * 8;
            if (rr >= rows) continue;
            RowCoord rcv;
            const long long r = row_voxel(rr, rcv);  // output row in the D x H x W space
#pragma unroll
            for (int nt = 0; nt < NT / 8; ++nt) {
                const int n = n0 + nt * 8 + tig * 2;
                if (n >= Nn) continue;
                float v0 = acc[mt][nt][half * 2], v1 = acc[mt][nt][half * 2 + 1];
                if (bias) {
                    v0 += bias[n];
                    if (n + 1 < Nn) v1 += bias[n + 1];
                }
                if (g.relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                if (g.mask) {  // ReLU derivative of the layer whose output is this gradient's tensor
                    const unsigned short *m = (const unsigned short *)g.mask + r * Nn + n;
                    if ((short)m[0] <= 0) v0 = 0.f;
                    if (n + 1 < Nn && (short)m[1] <= 0) v1 = 0.f;
                }
                if (out_f32) {
                    out_f32[r * Nn + n] = v0;
                    if (n + 1 < Nn) out_f32[r * Nn + n + 1] = v1;
                }
                if (out_bf16) {
                    if (n + 1 < Nn) {
                        *(__nv_bfloat162 *)(out_bf16 + r * Nn + n) = __floats2bfloat162_rn(v0, v1);
                    } else {
                        out_bf16[r * Nn + n] = __float2bfloat16_rn(v0);
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------- tcgen05
// 3x3x3 stride-1 padding-1 convolution on the fifth-generation tensor cores:
// a CTA of four warps owns a 1 x 16 x 8 block of output voxels (M = 128 rows,
// row m = 8 * (h - h0) + (w - w0)) and NT output channels.  Per 16-channel
// input slice it stages the 3 x 18 x 10 input halo and the slice's weights in
// shared memory in the canonical K-major layout without swizzle (8 rows of
// 16 bytes per core matrix), and one thread issues the 27 tap GEMMs
// (128 x NT x 16 each) as tcgen05.mma with the FP32 accumulator in tensor
// memory.  The halo is stored [d][h][k-chunk][w][8 channels], so the eight
// rows of a core matrix (eight consecutive w) are contiguous for any tap
// offset kw: the A operand of tap (kd, kh, kw) is the halo itself, seen
// through a descriptor at byte offset ((kd * 18 + kh) * 2) * 160 + kw * 16
// with 160 bytes between k-chunks and 320 bytes between rows of w.
// The input may be the channel concatenation of two tensors, src (ca channels,
// optionally at half resolution and read through nearest x2 upsampling) and
// src_b (cs - ca channels, full resolution), so that the decoder's upsampling
// and skip concatenation never materialise.  Every wait on the accumulator is
// bounded; on timeout the CTA records FDC_ERR_TIMEOUT in g_tc_status, skips
// its epilogue, frees its tensor memory and returns.
constexpr int kTcHD = 3, kTcHH = 18, kTcHW = 10;
constexpr int kTcHaloRows = kTcHD * kTcHH * kTcHW;             // 540 voxels
constexpr int kTcChunkBytes = kTcHW * 16;                      // one k-chunk of one (d, h) row: 160 B
constexpr int kTcHaloBytes = kTcHD * kTcHH * 2 * kTcChunkBytes;  // 17280 B
constexpr long long kTcWaitCycles = 4000000000ll;  // ~2 s at 2 GHz

__device__ int g_tc_status;  // FDC_ERR_TIMEOUT once an accumulator wait has timed out

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (no swizzle, K-major): start address,
// leading byte offset (between core matrices along K), stride byte offset
// (between groups of eight rows), all in 16-byte units; descriptor version 1.
__device__ __forceinline__ unsigned long long umma_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
    return (unsigned long long)((saddr >> 4) & 0x3fffu) | ((unsigned long long)((lbo >> 4) & 0x3fffu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 and M >> 4.
__host__ __device__ constexpr unsigned umma_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(unsigned tmem_d, unsigned long long a, unsigned long long b, unsigned idesc,
                                          int accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ bool mbar_wait_bounded(unsigned mbar, unsigned parity, long long limit = kTcWaitCycles) {
    const long long t0 = clock64();
    for (;;) {
        unsigned ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > limit) return false;
    }
}

// Test hook of the timeout path: one thread waits on an mbarrier that nothing
// completes, gives up after `cycles` and records FDC_ERR_TIMEOUT exactly as a
// convolution CTA would.
__global__ void wait_timeout_kernel(long long cycles) {
    __shared__ __align__(8) unsigned long long mbar;
    if (threadIdx.x != 0) return;
    const unsigned mb = smem_u32(&mbar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    if (!mbar_wait_bounded(mb, 0, cycles)) atomicExch(&g_tc_status, (int)FDC_ERR_TIMEOUT);
}

__device__ __forceinline__ void tmem_ld16(unsigned taddr, float v[16]) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld8(unsigned taddr, float v[8]) {
    unsigned r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                 "tcgen05.wait::ld.sync.aligned;\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Three 16-column loads (the kw blocks of a kw-stacked accumulator) with one
// wait: the loads overlap instead of each waiting in turn.
__device__ __forceinline__ void tmem_ld16x3(unsigned t0, unsigned t1, unsigned t2, float a[16], float b[16],
                                            float c[16]) {
    unsigned r[48];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%48];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, "
        "%29, %30, %31}, [%49];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, "
        "%45, %46, %47}, [%50];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
          "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
          "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47])
        : "r"(t0), "r"(t1), "r"(t2)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        a[i] = __uint_as_float(r[i]);
        b[i] = __uint_as_float(r[16 + i]);
        c[i] = __uint_as_float(r[32 + i]);
    }
}

// ReLU derivative of the previous layer, applied to a data-gradient output
// row: channels [n, n + 16) of voxel v become zero where that layer's output
// (the convolution's input, `mask`, Nn channels per voxel) is not positive.
// ReLU derivative of the previous layer on CW output channels of a
// data-gradient row (zero where that layer's output is not positive).
template <int CW>
__device__ __forceinline__ void apply_relu_mask(const void *mask, long long v, int Nn, int n, float a[CW]) {
    const uint4 *m = (const uint4 *)((const __nv_bfloat16 *)mask + v * Nn + n);
    uint4 q[CW / 8];
#pragma unroll
    for (int k = 0; k < CW / 8; ++k) q[k] = __ldg(m + k);
    const unsigned short *h = (const unsigned short *)q;
#pragma unroll
    for (int j = 0; j < CW; ++j)
        if ((short)h[j] <= 0) a[j] = 0.f;  // sign bit set, or +0: not positive
}

// Mask of output channels [n, n + CW) at voxel (b, d, h, w) of a D x H x W
// grid when the layer's forward input was [upsample?(a) | b] (g.mask_ca > 0).
template <int CW>
__device__ __forceinline__ void apply_relu_mask_fused(const Conv3dArgs &g, int Nn, int bb, int d, int h, int w, int D,
                                                      int H, int W, int n, float a[CW]) {
    const __nv_bfloat16 *m;
    if (n < g.mask_ca) {
        const long long vv = g.mask_up ? (((long long)bb * (D / 2) + (d >> 1)) * (H / 2) + (h >> 1)) * (W / 2) + (w >> 1)
                                       : (((long long)bb * D + d) * H + h) * W + w;
        m = (const __nv_bfloat16 *)g.mask + vv * g.mask_ca + n;
    } else {
        const long long vv = (((long long)bb * D + d) * H + h) * W + w;
        m = (const __nv_bfloat16 *)g.mask_b + vv * (Nn - g.mask_ca) + (n - g.mask_ca);
    }
    uint4 q[CW / 8];
#pragma unroll
    for (int k = 0; k < CW / 8; ++k) q[k] = __ldg((const uint4 *)m + k);
    const unsigned short *hh = (const unsigned short *)q;
#pragma unroll
    for (int j = 0; j < CW; ++j)
        if ((short)hh[j] <= 0) a[j] = 0.f;
}

__device__ __forceinline__ void tmem_ld8x3(unsigned t0, unsigned t1, unsigned t2, float a[8], float b[8], float c[8]) {
    unsigned r[24];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%24];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%25];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%26];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23])
        : "r"(t0), "r"(t1), "r"(t2)
        : "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        a[i] = __uint_as_float(r[i]);
        b[i] = __uint_as_float(r[8 + i]);
        c[i] = __uint_as_float(r[16 + i]);
    }
}

__device__ __forceinline__ void apply_relu_mask16(const void *mask, long long v, int Nn, int n, float a[16]) {
    const uint4 *m = (const uint4 *)((const __nv_bfloat16 *)mask + v * Nn + n);
    const uint4 q[2] = {__ldg(m), __ldg(m + 1)};
    const unsigned short *h = (const unsigned short *)q;
#pragma unroll
    for (int j = 0; j < 16; ++j)
        if ((short)h[j] <= 0) a[j] = 0.f;  // sign bit set, or +0: not positive
}

__device__ __forceinline__ void umma_commit(unsigned mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}

// 16 (h) x 8 (w) output voxels per CTA, 27 MMAs of N = NT per slice (NT = 64).
template <int NT>
__global__ void __launch_bounds__(128) conv3_tc_kernel(const Conv3dArgs g, const __nv_bfloat16 *src,
                                                       const __nv_bfloat16 *wt, const float *bias,
                                                       __nv_bfloat16 *out_bf16, float *out_f32, int Cs, int Nn,
                                                       int relu, int ca, int up_a, const __nv_bfloat16 *src_b) {
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *sH = smem;
    unsigned char *sW = smem + kTcHaloBytes;
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ unsigned tmem_slot;
    constexpr unsigned kCols = NT < 32 ? 32 : NT;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int D = g.in_d, H = g.in_h, W = g.in_w;
    const int tiles_w = (W + 7) / 8, tiles_h = (H + 15) / 16;
    long long t = blockIdx.x;
    const int tw = (int)(t % tiles_w); t /= tiles_w;
    const int th = (int)(t % tiles_h); t /= tiles_h;
    const int d0 = (int)(t % D);
    const int b = (int)(t / D);
    const int h0 = th * 16, w0 = tw * 8;
    const int n0 = blockIdx.y * NT;
    const int slices = Cs / 16;
    const int cb = Cs - ca;
    const int Da = up_a ? D / 2 : D, Ha = up_a ? H / 2 : H, Wa = up_a ? W / 2 : W;
    const unsigned mb = smem_u32(&mbar);

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const unsigned tmem = tmem_slot;

    bool ok = true;
    unsigned phase = 0;
    for (int sl = 0; sl < slices && ok; ++sl) {
        const int c0 = sl * 16;
        const bool from_a = c0 < ca;
        for (int i = tid; i < kTcHaloRows * 2; i += 128) {
            const int row = i >> 1, kc = i & 1;
            const int hd = row / (kTcHH * kTcHW), hh = (row / kTcHW) % kTcHH, hw = row % kTcHW;
            const int d = d0 - 1 + hd, h = h0 - 1 + hh, w = w0 - 1 + hw;
            const bool in = d >= 0 && d < D && h >= 0 && h < H && w >= 0 && w < W;
            const __nv_bfloat16 *p = src;
            if (in) {
                if (from_a) {
                    const int da = up_a ? d >> 1 : d, ha = up_a ? h >> 1 : h, wa = up_a ? w >> 1 : w;
                    p = src + ((((long long)b * Da + da) * Ha + ha) * Wa + wa) * ca + c0 + kc * 8;
                } else {
                    p = src_b + ((((long long)b * D + d) * H + h) * W + w) * cb + (c0 - ca) + kc * 8;
                }
            }
            cp_async16(sH + ((hd * kTcHH + hh) * 2 + kc) * kTcChunkBytes + hw * 16, p, in);
        }
        for (int i = tid; i < 27 * 2 * NT; i += 128) {
            const int n = i % NT, q = i / NT, kc = q & 1, tap = q >> 1;
            const int co = n0 + n;
            const bool in = co < Nn;
            const __nv_bfloat16 *p = in ? wt + ((long long)co * 27 + tap) * Cs + c0 + kc * 8 : wt;
            // every CTA reads the same slice of weights: through L1, not from L2 each time
            cp_async16_ca(sW + ((tap * 2 + kc) * NT + n) * 16, p, in);
        }
        cp_async_commit();
        cp_async_wait<0>();
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const unsigned ha = smem_u32(sH), wa = smem_u32(sW);
            constexpr unsigned idesc = umma_idesc(128, NT);
#pragma unroll 1
            for (int tap = 0; tap < 27; ++tap) {
                const int kd = tap / 9, kh = (tap / 3) % 3, kw = tap % 3;
                const unsigned long long ad =
                    umma_desc(ha + ((kd * kTcHH + kh) * 2) * kTcChunkBytes + kw * 16, kTcChunkBytes, 2 * kTcChunkBytes);
                const unsigned long long bd = umma_desc(wa + tap * 2 * NT * 16, NT * 16, 128);
                umma_bf16(tmem, ad, bd, idesc, (sl | tap) != 0);
            }
            umma_commit(mb);
        }
        ok = mbar_wait_bounded(mb, phase);
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        ok = __syncthreads_and(ok);
    }

    if (ok) {
        const int m = warp * 32 + lane;
        const int h = h0 + (m >> 3), w = w0 + (m & 7);
        const bool in = h < H && w < W;
        const long long v = (((long long)b * D + d0) * H + h) * W + w;
#pragma unroll
        for (int c = 0; c < NT; c += 16) {
            float acc[16];
            tmem_ld16(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c, acc);
            const int n = n0 + c;
            if (!in || n >= Nn) continue;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                float x = acc[j];
                if (bias) x += bias[n + j];
                if (relu) x = fmaxf(x, 0.f);
                acc[j] = x;
            }
            if (g.mask) apply_relu_mask16(g.mask, v, Nn, n, acc);
            if (out_f32) {
#pragma unroll
                for (int j = 0; j < 16; ++j) out_f32[v * Nn + n + j] = acc[j];
            }
            if (out_bf16) {
                uint4 q[2];
                unsigned *qq = (unsigned *)q;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    __nv_bfloat162 p2 = __floats2bfloat162_rn(acc[2 * j], acc[2 * j + 1]);
                    qq[j] = *(unsigned *)&p2;
                }
                uint4 *dst = (uint4 *)(out_bf16 + v * Nn + n);
                dst[0] = q[0];
                dst[1] = q[1];
            }
        }
    } else if (tid == 0) {
        atomicExch(&g_tc_status, (int)FDC_ERR_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kCols));
    }
}


// kw-stacked form (NT = 16 or 32): the three taps along w share one MMA.  A
// CTA owns 8 (h) x 14 (w) output voxels and NT channels; the A operand is the
// input halo itself, 8 rows of h x 16 columns of w (M = 128, row m = 16 h + w'
// for input column w0 - 1 + w'), and one MMA per (kd, kh) multiplies it by the
// weights of the three kw taps stacked along N (N = 3 NT, column kw NT + co):
//   D[m][kw NT + co] = sum_{kd, kh, ci} x[d0 - 1 + kd][h0 - 1 + h + kh][w0 - 1 + w'][ci]
//                                       * w[co][kd][kh][kw][ci],
// so that y[h][w][co] = sum_kw D[16 h + w + kw][kw NT + co]: 9 MMAs per 16-channel
// slice instead of 27, each three times wider (tensor-core time per MMA is
// dominated by its fixed part at N = 16).  The epilogue adds the three column
// blocks with lane shuffles (rows m + 1, m + 2 belong to lanes t + 1, t + 2 of
// the same warp).  Halo layout [d 3][h 10][w-group 2][k-chunk 2][8 w][8 ch]:
// 256 bytes per (d, h, w-group), so consecutive 8-row groups of A are 256
// bytes apart and k-chunks 128 bytes apart.
constexpr int kKwHD = 3, kKwHH = 10, kKwHW = 16;
constexpr int kKwHalo = kKwHD * kKwHH * kKwHW;  // 480 voxels
constexpr int kKwHaloBytes = kKwHalo * 32;      // 15360 B

// A CTA walks `tpc` consecutive output blocks of its NT-channel column; when
// the weights of all input slices fit (resw), they are staged once per CTA.
// Staging addresses are updated incrementally: in the halo loader every
// thread keeps one w column and one k-chunk and steps through (d, h) rows.
template <int NT>
__global__ void __launch_bounds__(128) conv3_kws_kernel(const Conv3dArgs g, const __nv_bfloat16 *src,
                                                        const __nv_bfloat16 *wt, const float *bias,
                                                        __nv_bfloat16 *out_bf16, float *out_f32, int Cs, int Nn,
                                                        int relu, int ca, int up_a, const __nv_bfloat16 *src_b,
                                                        int tpc, int resw) {
    constexpr int N3 = 3 * NT;
    constexpr unsigned kCols = N3 <= 64 ? 64 : 128;
    constexpr int kWChunks = 9 * 2 * N3;       // 16-byte chunks of one slice of weights
    constexpr int kWBytes = kWChunks * 16;
    constexpr int kQa = 128 / N3, kNa = 128 % N3;  // loader stride 128 in (q, n) digits
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *sH = smem;
    unsigned char *sW = smem + kKwHaloBytes;  // [slice][kd kh][k-chunk][kw NT + co][8]
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ unsigned tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int D = g.in_d, H = g.in_h, W = g.in_w;
    const int tiles_w = (W + 13) / 14, tiles_h = (H + 7) / 8;
    const long long n_tiles = (long long)g.batch * D * tiles_h * tiles_w;
    const int n0 = blockIdx.y * NT;
    const int slices = Cs / 16;
    const int cb = Cs - ca;
    const int Da = up_a ? D / 2 : D, Ha = up_a ? H / 2 : H, Wa = up_a ? W / 2 : W;
    const unsigned mb = smem_u32(&mbar);

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const unsigned tmem = tmem_slot;

    // weights of slice sl into sW + slot * kWBytes (through L1: every CTA reads the same)
    auto load_weights = [&](int sl, int slot) {
        int n = tid % N3, q = tid / N3;
        unsigned char *dst = sW + slot * kWBytes;
        for (int i = tid; i < kWChunks; i += 128) {
            const int kc = q & 1, kdh = q >> 1;
            const int co = n0 + (n % NT), kw = n / NT;
            const bool in = co < Nn;
            const __nv_bfloat16 *p = in ? wt + (size_t)((co * 27 + kdh * 3 + kw) * Cs + sl * 16 + kc * 8) : wt;
            cp_async16_ca(dst + i * 16, p, in);
            n += kNa;
            q += kQa;
            if (n >= N3) {
                n -= N3;
                ++q;
            }
        }
    };
    // this thread's halo column and k-chunk; rows r = d * 10 + h of the halo
    const int kc = tid & 1, hw = (tid >> 1) & 15, r0 = tid >> 5;
    const unsigned hdst = (unsigned)((((hw >> 3) * 2 + kc) * 128) + (hw & 7) * 16);

    if (resw)
        for (int sl = 0; sl < slices; ++sl) load_weights(sl, sl);

    bool ok = true;
    unsigned phase = 0;
    for (int it = 0; it < tpc && ok; ++it) {
        const long long tile = (long long)blockIdx.x * tpc + it;
        if (tile >= n_tiles) break;
        long long t = tile;
        const int w0 = (int)(t % tiles_w) * 14; t /= tiles_w;
        const int h0 = (int)(t % tiles_h) * 8; t /= tiles_h;
        const int d0 = (int)(t % D);
        const int b = (int)(t / D);
        const int w = w0 - 1 + hw;
        const bool w_in = w >= 0 && w < W;
        for (int sl = 0; sl < slices && ok; ++sl) {
            const int c0 = sl * 16;
            if (!resw) load_weights(sl, 0);
            const bool from_a = c0 < ca;
#pragma unroll 2
            for (int r = r0; r < kKwHD * kKwHH; r += 4) {
                const int hd = (r >= 10) + (r >= 20), hh = r - 10 * hd;
                const int d = d0 - 1 + hd, h = h0 - 1 + hh;
                const bool in = w_in && d >= 0 && d < D && h >= 0 && h < H;
                const __nv_bfloat16 *p = src;
                if (in) {
                    if (!from_a)
                        p = src_b + ((((long long)b * D + d) * H + h) * W + w) * cb + (c0 - ca) + kc * 8;
                    else if (up_a)
                        p = src + ((((long long)b * Da + (d >> 1)) * Ha + (h >> 1)) * Wa + (w >> 1)) * ca + c0 + kc * 8;
                    else
                        p = src + ((((long long)b * D + d) * H + h) * W + w) * ca + c0 + kc * 8;
                }
                cp_async16(sH + r * 512 + hdst, p, in);
            }
            cp_async_commit();
            cp_async_wait<0>();
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const unsigned ha = smem_u32(sH), wa = smem_u32(sW + (resw ? sl : 0) * kWBytes);
                constexpr unsigned idesc = umma_idesc(128, N3);
#pragma unroll 1
                for (int kdh = 0; kdh < 9; ++kdh) {
                    const int kd = kdh / 3, kh = kdh % 3;
                    const unsigned long long ad = umma_desc(ha + (kd * kKwHH + kh) * 512, 128, 256);
                    const unsigned long long bd = umma_desc(wa + kdh * 2 * N3 * 16, N3 * 16, 128);
                    umma_bf16(tmem, ad, bd, idesc, (sl | kdh) != 0);
                }
                umma_commit(mb);
            }
            // the MMAs read the halo (and a reloaded weight slice): wait before restaging
            ok = mbar_wait_bounded(mb, phase);
            phase ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            ok = __syncthreads_and(ok);
        }
        if (!ok) break;

        const int m = warp * 32 + lane;
        const int ho = h0 + (m >> 4), wl = m & 15, wo = w0 + wl;
        const bool out_in = wl < 14 && ho < H && wo < W;
        const long long v = (((long long)b * D + d0) * H + ho) * W + wo;
        const unsigned base = tmem + ((unsigned)(warp * 32) << 16);
#pragma unroll
        for (int c = 0; c < NT; c += 16) {
            float a0[16], a1[16], a2[16];
            tmem_ld16x3(base + (unsigned)c, base + (unsigned)(NT + c), base + (unsigned)(2 * NT + c), a0, a1, a2);
#pragma unroll
            for (int j = 0; j < 16; ++j)
                a0[j] += __shfl_down_sync(0xffffffffu, a1[j], 1) + __shfl_down_sync(0xffffffffu, a2[j], 2);
            const int n = n0 + c;
            if (!out_in || n >= Nn) continue;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                float x = a0[j];
                if (bias) x += __ldg(bias + n + j);
                if (relu) x = fmaxf(x, 0.f);
                a0[j] = x;
            }
            if (g.mask) apply_relu_mask16(g.mask, v, Nn, n, a0);
            if (out_f32) {
                float4 *dst = (float4 *)(out_f32 + v * Nn + n);
#pragma unroll
                for (int j = 0; j < 4; ++j) dst[j] = make_float4(a0[4 * j], a0[4 * j + 1], a0[4 * j + 2], a0[4 * j + 3]);
            }
            if (out_bf16) {
                uint4 q[2];
                unsigned *qq = (unsigned *)q;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    __nv_bfloat162 p2 = __floats2bfloat162_rn(a0[2 * j], a0[2 * j + 1]);
                    qq[j] = *(unsigned *)&p2;
                }
                uint4 *dst = (uint4 *)(out_bf16 + v * Nn + n);
                dst[0] = q[0];
                dst[1] = q[1];
            }
        }
        // every warp has read the accumulator before the next block's MMAs overwrite it
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    }
    if (!ok && tid == 0) atomicExch(&g_tc_status, (int)FDC_ERR_TIMEOUT);
    cp_async_wait<0>();
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kCols));
    }
}

// Epilogue of one output row of the d-walking kernels: CW output channels
// [n, n + CW) of voxel v = (b, d, ho, wo): bias (staged in shared memory,
// null for none), ReLU, the previous layer's ReLU mask of a data gradient
// (g.mask; split over two inputs when g.mask_ca > 0), and the store (FP32
// and/or BF16; with g.out_b, channels >= g.mask_ca go to the second output).
template <int CW>
__device__ __forceinline__ void dwalk_store(const Conv3dArgs &g, float a0[CW], const float *sb, int relu,
                                            __nv_bfloat16 *out_bf16, float *out_f32, int Nn, int n, int b, int d,
                                            int ho, int wo, long long v) {
#pragma unroll
    for (int j = 0; j < CW; ++j) {
        float x = a0[j];
        if (sb) x += sb[j];
        if (relu) x = fmaxf(x, 0.f);
        a0[j] = x;
    }
    if (g.mask) {
        if (g.mask_ca > 0)
            apply_relu_mask_fused<CW>(g, Nn, b, d, ho, wo, g.in_d, g.in_h, g.in_w, n, a0);
        else
            apply_relu_mask<CW>(g.mask, v, Nn, n, a0);
    }
    if (out_f32) {
        float4 *dst = (float4 *)(out_f32 + v * Nn + n);
#pragma unroll
        for (int j = 0; j < CW / 4; ++j) dst[j] = make_float4(a0[4 * j], a0[4 * j + 1], a0[4 * j + 2], a0[4 * j + 3]);
    }
    if (out_bf16) {
        uint4 qv[CW / 8];
        unsigned *qq = (unsigned *)qv;
#pragma unroll
        for (int j = 0; j < CW / 2; ++j) {
            __nv_bfloat162 p2 = __floats2bfloat162_rn(a0[2 * j], a0[2 * j + 1]);
            qq[j] = *(unsigned *)&p2;
        }
        // split output: channels >= mask_ca into out_b
        uint4 *dst = g.out_b == nullptr
                         ? (uint4 *)(out_bf16 + v * Nn + n)
                         : (n < g.mask_ca ? (uint4 *)(out_bf16 + v * g.mask_ca + n)
                                          : (uint4 *)((__nv_bfloat16 *)g.out_b + v * (Nn - g.mask_ca) + (n - g.mask_ca)));
#pragma unroll
        for (int j = 0; j < CW / 8; ++j) dst[j] = qv[j];
    }
}

// d-walking form of the kw-stacked convolution (input channels Cs <= 32,
// NT = 16 or 32 output channels per CTA): a CTA owns a contiguous range of
// output planes of one 8 (h) x 14 (w) column of tiles -- the flattened
// (tile, d) index space is split evenly over the CTAs, a range restarting at
// most once or twice at a tile boundary -- and walks it along d, so that each
// input plane of the column is staged once instead of three times.  Input
// planes (10 h x 16 w x Cs, layout [slice][h][w-group 2][k-chunk 2][8 w][8 ch],
// 5120 bytes per slice) live in a ring of R = PF + 4 slots and are fetched
// PF + 2 planes ahead of the output plane with cp.async (zero fill outside the
// grid); the weights of all input slices stay resident.  Output plane i of a
// range is computed by 9 * Cs / 16 MMAs (M = 128, N = 3 NT, K = 16) into one of
// two TMEM accumulators, and its epilogue (as in conv3_kws_kernel) runs while
// the MMAs of plane i + 1 execute.  Ring reuse: plane j overwrites plane
// j - R, last read by the MMAs of output plane j - R, whose completion was
// awaited two iterations before.  Every accumulator wait is bounded (on
// timeout: FDC_ERR_TIMEOUT, no further output, TMEM freed).
constexpr int kDwPlaneSliceBytes = 10 * 512;  // [h 10][w-group 2][k-chunk 2][8 w][8 ch]
#ifndef FDC_CONV_DWALK
#define FDC_CONV_DWALK 1
#endif
// widest input (channels) that takes the d-walking kernel; wider inputs use
// the kw-stacked kernel (the resident weights and a 5-plane ring must fit)
#ifndef FDC_CONV_DWALK_MAXC
#define FDC_CONV_DWALK_MAXC 64
#endif
// 64-channel output tiles (conv3_tc_kernel<64>) where they fill the GPU; the
// kw-stacked kernel's output tile width (0: 32 when the channels allow, 16: always 16)
#ifndef FDC_CONV_TC64
#define FDC_CONV_TC64 1
#endif
#ifndef FDC_KWS_NT
#define FDC_KWS_NT 16
#endif
// the d-walking kernel's shared memory at its smallest ring (5 planes) fits one CTA
inline bool dwalk_fits(int S, int NT) {
    return S * 9 * 2 * (3 * NT) * 16 + 5 * S * kDwPlaneSliceBytes <= 227 * 1024 - 1024;
}

// THR = 256: eight warps, warps w and w + 4 sharing an accumulator row
// quadrant (measured faster for 32-channel tiles and two-slice inputs);
// THR = 128 for one 16-channel input slice and 16-channel tiles (74 vs 82 us
// at 128^3).
template <int NT, int THR>
__global__ void __launch_bounds__(THR) conv3_dwalk_kernel(const Conv3dArgs g, const __nv_bfloat16 *src,
                                                          const __nv_bfloat16 *wt, const float *bias,
                                                          __nv_bfloat16 *out_bf16, float *out_f32, int Cs, int Nn,
                                                          int relu, int ca, int up_a, const __nv_bfloat16 *src_b,
                                                          int pf) {
    constexpr int N3 = 3 * NT;
    constexpr unsigned kAccCols = N3 <= 64 ? 64 : 128;  // columns per accumulator buffer
    constexpr unsigned kCols = 2 * kAccCols;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ unsigned tmem_slot;
    __shared__ float sBias[NT];  // the CTA's output channels are fixed: bias staged once
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int D = g.in_d, H = g.in_h, W = g.in_w;
    const int S = Cs / 16;
    const int R = pf + 4;
    const int plane_bytes = S * kDwPlaneSliceBytes;
    const int wbytes = S * 9 * 2 * N3 * 16;
    unsigned char *sW = smem;                // [slice][kd kh][k-chunk][kw NT + co][8]
    unsigned char *sP = smem + wbytes;       // R plane slots
    const int tiles_w = (W + 13) / 14, tiles_h = (H + 7) / 8;
    const long long n_cols = (long long)g.batch * tiles_h * tiles_w;
    const long long total = n_cols * D;      // (tile column, d) output planes
    const long long q_begin = total * blockIdx.x / gridDim.x, q_end = total * (blockIdx.x + 1) / gridDim.x;
    const int n0 = blockIdx.y * NT;
    const int cb = Cs - ca;
    const int Da = up_a ? D / 2 : D, Ha = up_a ? H / 2 : H, Wa = up_a ? W / 2 : W;
    const unsigned mb0 = smem_u32(&mbar[0]), mb1 = smem_u32(&mbar[1]);

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb1));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid < NT) sBias[tid] = (bias && n0 + tid < Nn) ? bias[n0 + tid] : 0.f;
    // resident weights of every input slice (through L1: all CTAs read the same)
    {
        constexpr int kChunks = 9 * 2 * N3;  // per slice
        for (int i = tid; i < S * kChunks; i += THR) {
            const int sl = i / kChunks, r = i % kChunks;
            const int n = r % N3, q = r / N3, kc = q & 1, kdh = q >> 1;
            const int co = n0 + (n % NT), kw = n / NT;
            const bool in = co < Nn;
            const __nv_bfloat16 *p = in ? wt + (size_t)((co * 27 + kdh * 3 + kw) * Cs + sl * 16 + kc * 8) : wt;
            cp_async16_ca(sW + i * 16, p, in);
        }
        cp_async_commit();
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const unsigned tmem = tmem_slot;

    // this thread's halo column and k-chunk; it walks rows r = slice * 10 + h
    constexpr int kRowStep = THR / 32;
    const int kc = tid & 1, hw = (tid >> 1) & 15, r0 = tid >> 5;
    const unsigned hdst = (unsigned)((((hw >> 3) * 2 + kc) * 128) + (hw & 7) * 16);
    bool ok = true;
    unsigned it_all = 0;  // iterations over all ranges: accumulator buffer and barrier phase
    for (long long q = q_begin; q < q_end && ok;) {
        const long long col = q / D;
        const int d_begin = (int)(q % D);
        const int nd = (int)(q_end - q < (long long)(D - d_begin) ? q_end - q : (long long)(D - d_begin));
        q += nd;
        long long t = col;
        const int w0 = (int)(t % tiles_w) * 14; t /= tiles_w;
        const int h0 = (int)(t % tiles_h) * 8;
        const int b = (int)(t / tiles_h);
        const int w = w0 - 1 + hw;
        const bool w_in = w >= 0 && w < W;
        // stage input plane j (= d_begin - 1 + j) into slot j % R, one commit group
        auto load_plane = [&](int j) {
            if (j <= nd + 1) {
                const int d = d_begin - 1 + j;
                unsigned char *dst = sP + (j % R) * plane_bytes + hdst;
                const bool d_in = w_in && d >= 0 && d < D;
                for (int r = r0; r < S * 10; r += kRowStep) {
                    const int sl = r / 10, hh = r - 10 * sl;
                    const int h = h0 - 1 + hh, c0 = sl * 16;
                    const bool in = d_in && h >= 0 && h < H;
                    const __nv_bfloat16 *p = src;
                    if (in) {
                        if (c0 >= ca)
                            p = src_b + ((((long long)b * D + d) * H + h) * W + w) * cb + (c0 - ca) + kc * 8;
                        else if (up_a)
                            p = src + ((((long long)b * Da + (d >> 1)) * Ha + (h >> 1)) * Wa + (w >> 1)) * ca + c0 +
                                kc * 8;
                        else
                            p = src + ((((long long)b * D + d) * H + h) * W + w) * ca + c0 + kc * 8;
                    }
                    cp_async16(dst + r * 512, p, in);
                }
            }
            cp_async_commit();
        };
        for (int j = 0; j < pf + 2; ++j) load_plane(j);
        int slot_i = 0;  // ring slot of input plane i (= i % R), advanced per output plane
        // epilogue of output plane i of this range (accumulator buffer ab, barrier phase ph)
        auto epilogue = [&](int i, unsigned ab, unsigned ph) -> bool {
            // warp-uniform outcome (the shuffles below need every lane)
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(ab ? mb1 : mb0, ph))) return false;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            // warp w reads the accumulator rows of lane quadrant w % 4; with eight
            // warps, w and w + 4 take output channels [0, NT/2) and [NT/2, NT)
            constexpr int CW = NT * 128 / THR;
            static_assert(CW == 8 || CW == 16, "8 or 16 output channels per thread");
            const int quad = warp & 3, c = (warp >> 2) * CW;
            const int m = quad * 32 + lane;
            const int ho = h0 + (m >> 4), wl = m & 15, wo = w0 + wl;
            const bool out_in = wl < 14 && ho < H && wo < W;
            const long long v = (((long long)b * D + d_begin + i) * H + ho) * W + wo;
            const unsigned base = tmem + ((unsigned)(quad * 32) << 16) + ab * kAccCols;
            float a0[CW], a1[CW], a2[CW];
            if constexpr (CW == 16)
                tmem_ld16x3(base + (unsigned)c, base + (unsigned)(NT + c), base + (unsigned)(2 * NT + c), a0, a1, a2);
            else
                tmem_ld8x3(base + (unsigned)c, base + (unsigned)(NT + c), base + (unsigned)(2 * NT + c), a0, a1, a2);
#pragma unroll
            for (int j = 0; j < CW; ++j)
                a0[j] += __shfl_down_sync(0xffffffffu, a1[j], 1) + __shfl_down_sync(0xffffffffu, a2[j], 2);
            const int n = n0 + c;
            if (out_in && n < Nn)
                dwalk_store<CW>(g, a0, bias ? sBias + c : nullptr, relu, out_bf16, out_f32, Nn, n, b, d_begin + i, ho,
                                wo, v);
            // every warp has read this accumulator before MMAs overwrite it
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            return true;
        };
        for (int i = 0; i < nd; ++i) {
            load_plane(i + pf + 2);
            // planes i, i + 1, i + 2 of the range are in shared memory (the
            // pf most recent groups may still be in flight)
            switch (pf) {  // all but the pf most recent plane groups have landed
                case 1: cp_async_wait<1>(); break;
                case 2: cp_async_wait<2>(); break;
                case 3: cp_async_wait<3>(); break;
                case 4: cp_async_wait<4>(); break;
                case 5: cp_async_wait<5>(); break;
                case 6: cp_async_wait<6>(); break;
                default: cp_async_wait<0>(); break;
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            // also agrees on the outcome of the previous epilogue's bounded wait
            if (!__syncthreads_and(ok)) {
                ok = false;
                break;
            }
            const unsigned ab = it_all & 1u;
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                constexpr unsigned idesc = umma_idesc(128, N3);
                // descriptors of the three input planes and of the weights; the
                // per-MMA offsets are added to the 16-byte address field (shared
                // addresses stay below 2^18, so the 14-bit field cannot carry)
                unsigned long long ad_kd[3];
#pragma unroll
                for (int kd = 0; kd < 3; ++kd) {
                    int sk = slot_i + kd;
                    if (sk >= R) sk -= R;
                    ad_kd[kd] = umma_desc(smem_u32(sP) + sk * plane_bytes, 128, 256);
                }
                const unsigned long long bd0 = umma_desc(smem_u32(sW), N3 * 16, 128);
#pragma unroll 1
                for (int sl = 0; sl < S; ++sl) {
#pragma unroll
                    for (int kdh = 0; kdh < 9; ++kdh) {
                        const unsigned long long ad =
                            ad_kd[kdh / 3] + (unsigned long long)((sl * kDwPlaneSliceBytes + (kdh % 3) * 512) >> 4);
                        const unsigned long long bd = bd0 + (unsigned long long)(((sl * 9 + kdh) * 2 * N3 * 16) >> 4);
                        umma_bf16(tmem + ab * kAccCols, ad, bd, idesc, (sl | kdh) != 0);
                    }
                }
                umma_commit(ab ? mb1 : mb0);
            }
            if (i > 0) ok = epilogue(i - 1, ab ^ 1u, ((it_all - 1) >> 1) & 1u);
            ++it_all;
            if (++slot_i == R) slot_i = 0;
        }
        // the range's last plane
        if (__syncthreads_and(ok)) ok = epilogue(nd - 1, (it_all - 1) & 1u, ((it_all - 1) >> 1) & 1u);
        else ok = false;
        ok = __syncthreads_and(ok);
        cp_async_wait<0>();
        __syncthreads();
    }
    if (!ok && tid == 0) atomicExch(&g_tc_status, (int)FDC_ERR_TIMEOUT);
    cp_async_wait<0>();
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kCols));
    }
}

// ---- d-walking convolution with TMA staging and warp roles
// The tiles, resident weights, kw-stacked MMAs and two TMEM accumulators of
// conv3_dwalk_kernel, for inputs read as stored ([a | b] at one resolution,
// split at a 16-channel slice boundary).  Each input plane arrives by TMA: per
// 16-channel slice one 5-D box (16 channels x 16 w x 10 h x 1 d x 1 batch,
// zero fill outside the grid) written with the 32-byte swizzle, which is the
// canonical SWIZZLE_32B K-major operand layout (rows of 32 B, eight-row groups
// 256 B apart), so an MMA reads the A tile of tap kh at row 16 kh of the plane
// directly and no thread computes a staging address.  Warp roles hand off
// through mbarriers only (no CTA barrier inside the walk):
//   full[s]   TMA warp -> MMA warp: the plane in ring slot s has landed
//   empty[s]  MMA warp -> TMA warp: the MMAs that read slot s have completed
//   accf[k]   MMA warp -> epilogue: accumulator k holds an output plane
//   acce[k]   epilogue -> MMA warp: all EW epilogue warps have read it
// Warps 0..EW-1 run the epilogue (TMEM lane quadrant warp % 4; with EW = 8
// warps w and w + 4 take the two halves of the output channels), warp EW
// issues the TMA copies, warp EW + 1 the MMAs.  Input plane j of a range is
// read by output planes j - 2 .. j and released after output plane j.
// Every wait is bounded: an expired wait records FDC_ERR_TIMEOUT and raises a
// CTA-wide abort flag that ends the other roles' waits; before TMEM is freed
// the TMA warp waits (bounded) for the copies it issued and the MMA warp for
// its MMAs.
constexpr int kDwtMaxRing = 12;
constexpr int kDwtMaxAcc = 8;   // accumulator slots
// the K dimension of inputs wider than 64 channels split over CTAs
#ifndef FDC_DWT_KSPLIT
#define FDC_DWT_KSPLIT 1
#endif
// input channels per K part of a split layer (32 or 64)
#ifndef FDC_DWT_KSPLIT_CH
#define FDC_DWT_KSPLIT_CH 64
#endif
// pair tiles (MODE 2) for inputs made of two 16-channel tensors
#ifndef FDC_DWT_PAIR
#define FDC_DWT_PAIR 1
#endif
#ifndef FDC_CONV_DWTMA
#define FDC_CONV_DWTMA 1
#endif

__device__ __forceinline__ bool mbar_try(unsigned mb, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mb), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of parity `parity` of barrier mb; false when the CTA's
// abort flag is raised or the wait expires (which raises the flag).
__device__ __forceinline__ bool role_wait(unsigned mb, unsigned parity, volatile int *abort_flag) {
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try(mb, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > kTcWaitCycles) {
            *abort_flag = 1;
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_5d(unsigned dst, const void *tmap, int c0, int c1, int c2, int c3, int c4,
                                            unsigned mb) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5, %6}], [%7];\n" ::"r"(dst),
        "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(mb)
        : "memory");
}

// Shared-memory matrix descriptor, K-major with the 32-byte swizzle: rows of
// 32 B (16 BF16, one MMA's K), eight-row groups `sbo` bytes apart (the
// leading offset is unused: K fits in one swizzle atom); version 1, layout 6.
__device__ __forceinline__ unsigned long long umma_desc_sw32(unsigned saddr, unsigned sbo) {
    return (unsigned long long)((saddr >> 4) & 0x3fffu) | (1ull << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46) | (6ull << 61);
}

// MODE 1: the convolution of the nearest x2 upsampling of the input,
// computed on the input's own (coarse) grid by output parity class
// (sub-pixel form): along an axis, output 2i + p reads coarse voxels
// i + p - 1 + s' (s' = 0, 1) with the weights of the taps that land there
// summed (p = 0: tap 0 | taps 1, 2; p = 1: taps 0, 1 | tap 2), so each output
// voxel takes 8 collapsed taps instead of 27.  A coarse output plane is four
// units (pd, ph); a unit is 4 (sd', sh') MMAs per 16-channel slice whose N =
// 4 NT columns hold the blocks (pw, sw') of the w axis, added in the epilogue
// like the kw blocks of MODE 0.  Weights: fdc's collapsed layout
// [c_out][pd ph][sd' sh'][pw sw'][c_in] (conv3_collapse_up_kernel).
// MODE 2 (inputs made of 16-channel tensors, even w): pair tiles.  Each
// 64-byte row of a plane holds two neighbouring voxels' 16 channels (one TMA
// box per tensor: 32 values x 16 voxel pairs x 10 h, 64-byte swizzle), so a
// box fetches 32 input columns in rows of 64 B instead of 16 columns in rows
// of 32 B; the MMAs of a (kd, kh) tap read the even (e = 0) and the odd
// (e = 1) voxel of every pair as two K-major A operands 32 B apart in the
// swizzle atom, into two accumulators D_e, D_o.  A tile's first output column
// is w0 = 30 t - 1; it loads columns w0 - 1 .. w0 + 30 and yields w0 ..
// w0 + 29: pair P (columns w0 - 1 + 2P, w0 + 2P) gives
//   w0 + 2P     = D_e[P] kw0 + D_o[P] kw1 + D_e[P+1] kw2,
//   w0 + 2P + 1 = D_o[P] kw0 + D_e[P+1] kw1 + D_o[P+1] kw2.
// The same with the 64-byte swizzle (rows of 64 B, eight-row groups `sbo`
// bytes apart; layout 4); a start address 32 B into a row selects its second
// 16 BF16 as the K slice.
__device__ __forceinline__ unsigned long long umma_desc_sw64(unsigned saddr, unsigned sbo) {
    return (unsigned long long)((saddr >> 4) & 0x3fffu) | (1ull << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46) | (4ull << 61);
}

// MODE 3: the data gradient of the MODE 1 convolution, on the coarse grid:
// da[m] = sum over output parities q and coarse offsets of Wc^T dy[2 (m + o) + q],
// o in {0, +1} for q = 0 and {-1, 0} for q = 1 per axis (the adjoint of the
// collapse: the offset index idx = o for q = 0, o + 1 for q = 1 takes the
// collapsed weights of s' = 1 - idx).  The ring holds full-resolution dy planes,
// each as four boxes of its (h, w) parity classes (TMA element stride 2 in w
// and h: 16 coarse columns x 10 coarse rows); coarse output plane i reads
// full-resolution planes 2i - 1 .. 2i + 2 (two new ones per output).  Per
// (q, idx_d, idx_h) one MMA of N = 2 NT (the two w offsets) into the
// accumulator half of q_w; the epilogue adds the four w blocks with lane
// shuffles and applies the ReLU mask of a (coarse).  Weights: the transposed
// collapsed layout [c_a][64][c_out] (conv3_collapse_up_t_kernel).
template <int NT, int EW, int MINB, int MODE>
__global__ void __launch_bounds__(32 * (EW + 2), MINB)
    conv3_dwtma_kernel(const __grid_constant__ CUtensorMap tm_a, const __grid_constant__ CUtensorMap tm_b,
                       const Conv3dArgs g, const __nv_bfloat16 *wt, const float *bias, __nv_bfloat16 *out_bf16,
                       float *out_f32, int Cs, int Nn, int relu, int ca, int R, int NA, int cw,
                       long long split_stride) {
    // K split over blockIdx.z: this CTA's input channels are [c_off, c_off + Cs) of
    // the cw channels of the weights; its FP32 partial sums go to out_f32 + z * split_stride
    const int c_off = (int)blockIdx.z * Cs;
    if (gridDim.z > 1) out_f32 += (long long)blockIdx.z * split_stride;
    // column blocks per MMA: kw taps | (pw, sw') | kw taps | the two w offsets of a parity
    constexpr int NB = MODE == 1 ? 4 : (MODE == 3 ? 2 : 3);
    // weight groups per slice: (kd, kh) | (pd ph, sd' sh') | (kd, kh) | (q, idx_d, idx_h)
    constexpr int NU = MODE == 1 ? 16 : (MODE == 3 ? 32 : 9);
    constexpr int NX = NB * NT;                    // MMA N
    // columns per accumulator slot (MODE 2: D_e and D_o, 64 apart; MODE 3: the two w parities)
    constexpr unsigned kAccCols = MODE == 2 ? 128 : (MODE == 3 ? 4 * NT : (NX <= 64 ? 64 : 128));
    constexpr int UPP = MODE == 1 ? 4 : 1;         // units per (coarse) output plane
    constexpr int kPPO = MODE == 3 ? 2 : 1;        // new input planes per output plane
    constexpr int kSpan = MODE == 3 ? 4 : 3;       // input planes one output plane reads
    constexpr int kBoxes = MODE == 3 ? 4 : 1;      // boxes per slice of an input plane
    // bytes per slice of a plane (all of its boxes)
    constexpr int kSlice = MODE == 2 ? 2 * kDwPlaneSliceBytes : kBoxes * kDwPlaneSliceBytes;
    constexpr int kTileW = MODE == 2 ? 30 : 14;    // output columns per tile
    static_assert(MODE != 2 || (NT == 16 && EW == 8), "pair tiles: 16-channel output tiles, 8 epilogue warps");
    constexpr int THR = 32 * (EW + 2);
    constexpr int kMmaWarp = EW + 1;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long bars[2 * kDwtMaxRing + 2 * kDwtMaxAcc + 1];
    __shared__ unsigned tmem_slot;
    __shared__ int abort_flag;
    __shared__ float sBias[NT];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // the walked grid: the output grid (MODE 0, 2) or the coarse grid (MODE 1, 3)
    constexpr bool kCoarse = MODE == 1 || MODE == 3;
    const int D = kCoarse ? g.in_d / 2 : g.in_d, H = kCoarse ? g.in_h / 2 : g.in_h,
              W = kCoarse ? g.in_w / 2 : g.in_w;
    const int S = Cs / 16;
    const unsigned plane_bytes = (unsigned)(S * kSlice);
    const int wbytes = S * NU * 2 * NX * 16;
    const unsigned kCols = (unsigned)NA * kAccCols;
    unsigned char *sW = smem;  // [slice][group][k-chunk][block NT + co][8]
    // the plane ring starts on a 1024-byte boundary (the swizzle pattern is
    // taken from the shared-memory address bits)
    const unsigned sP = (smem_u32(smem) + (unsigned)wbytes + 1023u) & ~1023u;
    const unsigned bar0 = smem_u32(&bars[0]);
    auto full = [&](int s) { return bar0 + 8u * (unsigned)s; };
    auto empty = [&](int s) { return bar0 + 8u * (unsigned)(kDwtMaxRing + s); };
    auto accf = [&](unsigned k) { return bar0 + 8u * (2u * kDwtMaxRing + k); };
    auto acce = [&](unsigned k) { return bar0 + 8u * (2u * kDwtMaxRing + kDwtMaxAcc + k); };
    const unsigned fin = bar0 + 8u * (2u * kDwtMaxRing + 2u * kDwtMaxAcc);
    volatile int *abort_v = &abort_flag;

    // MODE 2 tiles start 2 columns before their first output (the first tile at w = -1)
    const int tiles_w = MODE == 2 ? (W + 1 + kTileW - 1) / kTileW : (W + kTileW - 1) / kTileW, tiles_h = (H + 7) / 8;
    const long long n_cols = (long long)g.batch * tiles_h * tiles_w;
    const long long total = n_cols * D;  // (tile column, d) output planes
    const long long q_begin = total * blockIdx.x / gridDim.x, q_end = total * (blockIdx.x + 1) / gridDim.x;
    const int n0 = blockIdx.y * NT;

    if (tid == 0) {
        for (int s = 0; s < R; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(full(s)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(empty(s)));
        }
        for (unsigned k = 0; k < (unsigned)NA; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(accf(k)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(acce(k)), "r"(EW));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(fin));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        abort_flag = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid < NT) sBias[tid] = (bias && n0 + tid < Nn) ? bias[n0 + tid] : 0.f;
    {  // resident weights of every input slice (through L1: all CTAs read the same)
        constexpr int kChunks = NU * 2 * NX;  // per slice
        constexpr int kTaps = MODE == 1 || MODE == 3 ? 64 : 27;  // weight rows per output channel
        for (int i = tid; i < S * kChunks; i += THR) {
            const int sl = i / kChunks, r = i % kChunks;
            const int n = r % NX, q = r / NX, kc = q & 1, grp = q >> 1;
            const int co = n0 + (n % NT), blk = n / NT;
            const bool in = co < Nn;
            const __nv_bfloat16 *p =
                in ? wt + (size_t)((co * kTaps + grp * NB + blk) * cw + c_off + sl * 16 + kc * 8) : wt;
            cp_async16_ca(sW + i * 16, p, in);
        }
        cp_async_commit();
        cp_async_wait<0>();
    }
    // weights written by the generic proxy are read by the MMAs (async proxy)
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const unsigned tmem = tmem_slot;

    // the (tile column, d) ranges of this CTA, identical for every role
    auto range_at = [&](long long q, int &d_begin, int &nd, int &w0, int &h0, int &b) {
        const long long col = q / D;
        d_begin = (int)(q % D);
        nd = (int)(q_end - q < (long long)(D - d_begin) ? q_end - q : (long long)(D - d_begin));
        long long t = col;
        w0 = (int)(t % tiles_w) * kTileW - (MODE == 2 ? 1 : 0);  // first output column
        t /= tiles_w;
        h0 = (int)(t % tiles_h) * 8;
        b = (int)(t / tiles_h);
    };

    if (warp == EW) {  // ---- TMA: stage input planes d_begin - 1 .. d_begin + nd of each range
        if (lane == 0) {
            unsigned p = 0;  // planes issued over all ranges (ring slot p % R)
            bool ok = true;
            for (long long q = q_begin; q < q_end && ok;) {
                int d_begin, nd, w0, h0, b;
                range_at(q, d_begin, nd, w0, h0, b);
                q += nd;
                for (int j = 0; j < kPPO * nd + kSpan - kPPO; ++j, ++p) {
                    const int s = (int)(p % (unsigned)R);
                    if (p >= (unsigned)R && !role_wait(empty(s), (p / (unsigned)R - 1u) & 1u, abort_v)) {
                        ok = false;
                        break;
                    }
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(full(s)),
                                 "r"(plane_bytes)
                                 : "memory");
                    // MODE 3: full-resolution planes 2 d_begin - 1 + j, four parity boxes per slice
                    const int d = MODE == 3 ? 2 * d_begin - 1 + j : d_begin - 1 + j;
                    if constexpr (MODE == 3) {
                        for (int bx = 0; bx < 4; ++bx)
                            for (int sl = 0; sl < S; ++sl) {
                                const unsigned dst =
                                    sP + (unsigned)s * plane_bytes + (unsigned)((bx * S + sl) * kDwPlaneSliceBytes);
                                tma_load_5d(dst, &tm_a, c_off + sl * 16, 2 * (w0 - 1) + (bx & 1),
                                            2 * (h0 - 1) + (bx >> 1), d, b, full(s));
                            }
                    } else {
                        for (int sl = 0; sl < S; ++sl) {
                            const unsigned dst = sP + (unsigned)s * plane_bytes + (unsigned)(sl * kSlice);
                            const int cg = c_off + sl * 16;  // the slice's first channel of [a | b]
                            if (MODE == 2)  // one 16-channel tensor per slice, columns w0 - 1 .. w0 + 30 as pairs
                                tma_load_5d(dst, sl == 0 ? (const void *)&tm_a : (const void *)&tm_b, 0,
                                            (w0 - 1) / 2, h0 - 1, d, b, full(s));
                            else if (cg < ca)
                                tma_load_5d(dst, &tm_a, cg, w0 - 1, h0 - 1, d, b, full(s));
                            else
                                tma_load_5d(dst, &tm_b, cg - ca, w0 - 1, h0 - 1, d, b, full(s));
                        }
                    }
                }
            }
            // copies still in flight land before the CTA exits (bounded)
            const unsigned n_out = p < (unsigned)R ? p : (unsigned)R;
            const long long t0 = clock64();
            for (unsigned pp = p - n_out; pp < p; ++pp)
                while (!mbar_try(full((int)(pp % (unsigned)R)), (pp / (unsigned)R) & 1u))
                    if (clock64() - t0 > kTcWaitCycles) break;
        }
        __syncwarp();
    } else if (warp == kMmaWarp) {  // ---- MMA: output units of each range
        if (lane == 0) {
            constexpr unsigned idesc = umma_idesc(128, NX);
            const unsigned long long bd0 = umma_desc(smem_u32(sW), NX * 16, 128);
            unsigned p = 0, it = 0;  // first plane of the range; units over all ranges
            bool ok = true;
            for (long long q = q_begin; q < q_end && ok;) {
                int d_begin, nd, w0, h0, b;
                range_at(q, d_begin, nd, w0, h0, b);
                q += nd;
                for (int i = 0; i < nd && ok; ++i) {
                    // output plane i reads input planes kPPO i .. kPPO i + kSpan - 1 of the range
                    for (int j = (i == 0 ? 0 : kPPO * i + kSpan - kPPO); j < kPPO * i + kSpan; ++j) {
                        const unsigned pp = p + (unsigned)j;
                        if (!role_wait(full((int)(pp % (unsigned)R)), (pp / (unsigned)R) & 1u, abort_v)) ok = false;
                    }
                    if (!ok) break;
                    unsigned long long ad_kd[kSpan];
#pragma unroll
                    for (int kd = 0; kd < kSpan; ++kd) {
                        const unsigned a = sP + ((p + (unsigned)(kPPO * i + kd)) % (unsigned)R) * plane_bytes;
                        ad_kd[kd] = MODE == 2 ? umma_desc_sw64(a, 512) : umma_desc_sw32(a, 256);
                    }
                    for (int u = 0; u < UPP; ++u, ++it) {
                        const unsigned ab = it % (unsigned)NA;
                        if (it >= (unsigned)NA && !role_wait(acce(ab), (it / (unsigned)NA - 1u) & 1u, abort_v)) {
                            ok = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll 1
                        for (int sl = 0; sl < S; ++sl) {
                            if constexpr (MODE == 3) {
                                // parity q = (qd, qh, qw), offsets (idx_d, idx_h): full-resolution plane
                                // 2i + 2 idx_d + 1 - qd of the range, row shift idx_h + 1 - qh,
                                // accumulator half qw
#pragma unroll
                                for (int grp = 0; grp < 32; ++grp) {
                                    const int qd = grp >> 4, qh = (grp >> 3) & 1, qw = (grp >> 2) & 1,
                                              idd = (grp >> 1) & 1, idh = grp & 1;
                                    const int f = 2 * idd + 1 - qd, kh = idh + 1 - qh, bx = qh * 2 + qw;
                                    const unsigned long long ad =
                                        ad_kd[f] +
                                        (unsigned long long)(((bx * S + sl) * kDwPlaneSliceBytes + kh * 512) >> 4);
                                    const unsigned long long bd =
                                        bd0 + (unsigned long long)(((sl * NU + grp) * 2 * NX * 16) >> 4);
                                    umma_bf16(tmem + ab * kAccCols + (unsigned)(qw * NX), ad, bd, idesc,
                                              (sl | qd | qh | idd | idh) != 0);
                                }
                            } else if constexpr (MODE == 2) {
                                // tap (kd, kh): the even and the odd voxel of every pair (rows of
                                // 64 B, 16 pairs per h row: kh shifts by 1 KB, e by 32 B)
#pragma unroll
                                for (int kdh = 0; kdh < 9; ++kdh) {
                                    const unsigned long long bd =
                                        bd0 + (unsigned long long)(((sl * NU + kdh) * 2 * NX * 16) >> 4);
#pragma unroll
                                    for (int e = 0; e < 2; ++e) {
                                        const unsigned long long ad =
                                            ad_kd[kdh / 3] +
                                            (unsigned long long)((sl * kSlice + (kdh % 3) * 1024 + e * 32) >> 4);
                                        umma_bf16(tmem + ab * kAccCols + (unsigned)(e * 64), ad, bd, idesc,
                                                  (sl | kdh) != 0);
                                    }
                                }
                            } else if constexpr (MODE == 0) {
#pragma unroll
                                for (int kdh = 0; kdh < 9; ++kdh) {
                                    const unsigned long long ad =
                                        ad_kd[kdh / 3] +
                                        (unsigned long long)((sl * kDwPlaneSliceBytes + (kdh % 3) * 512) >> 4);
                                    const unsigned long long bd =
                                        bd0 + (unsigned long long)(((sl * NU + kdh) * 2 * NX * 16) >> 4);
                                    umma_bf16(tmem + ab * kAccCols, ad, bd, idesc, (sl | kdh) != 0);
                                }
                            } else {
                                // unit u = (pd, ph); combination c = (sd', sh') reads input
                                // plane i + pd + sd' - 1 (ring index pd + sd') at row shift ph + sh'
                                const int pd = u >> 1, ph = u & 1;
#pragma unroll
                                for (int c = 0; c < 4; ++c) {
                                    const int kd = pd + (c >> 1), kh = ph + (c & 1);
                                    const unsigned long long ad =
                                        ad_kd[kd] + (unsigned long long)((sl * kDwPlaneSliceBytes + kh * 512) >> 4);
                                    const unsigned long long bd =
                                        bd0 + (unsigned long long)(((sl * NU + u * 4 + c) * 2 * NX * 16) >> 4);
                                    umma_bf16(tmem + ab * kAccCols, ad, bd, idesc, (sl | c) != 0);
                                }
                            }
                        }
                        umma_commit(accf(ab));
                    }
                    if (!ok) break;
                    for (int j = 0; j < kPPO; ++j)  // input planes this output plane read last
                        umma_commit(empty((int)((p + (unsigned)(kPPO * i + j)) % (unsigned)R)));
                }
                if (!ok) break;
                // the range's last input planes are released after its last MMAs
                for (int j = kPPO * nd; j < kPPO * nd + kSpan - kPPO; ++j)
                    umma_commit(empty((int)((p + (unsigned)j) % (unsigned)R)));
                p += (unsigned)(kPPO * nd + kSpan - kPPO);
            }
            // every MMA issued has completed before TMEM is freed (bounded)
            umma_commit(fin);
            const long long t0 = clock64();
            while (!mbar_try(fin, 0))
                if (clock64() - t0 > kTcWaitCycles) break;
        }
        __syncwarp();
    } else {  // ---- epilogue warps
        constexpr int CW = NT * 128 / (32 * EW);
        static_assert(CW == 8 || CW == 16, "8 or 16 output channels per thread");
        const int quad = warp & 3, c = (warp >> 2) * CW;
        const int m = quad * 32 + lane;
        unsigned it = 0;
        bool ok = true;
        for (long long q = q_begin; q < q_end && ok;) {
            int d_begin, nd, w0, h0, b;
            range_at(q, d_begin, nd, w0, h0, b);
            q += nd;
            const int hl = h0 + (m >> 4), wl = m & 15, wc = w0 + wl;
            const bool out_in = wl < 14 && hl < H && wc < W;  // MODE 0, 1, 3
            for (int i = 0; i < nd && ok; ++i) {
                for (int u = 0; u < UPP; ++u, ++it) {
                    const unsigned ab = it % (unsigned)NA;
                    // warp-uniform outcome (the shuffles below need every lane)
                    if (!__all_sync(0xffffffffu, role_wait(accf(ab), (it / (unsigned)NA) & 1u, abort_v))) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const unsigned base = tmem + ((unsigned)(quad * 32) << 16) + ab * kAccCols;
                    const int n = n0 + c;
                    if constexpr (MODE == 3) {
                        // w blocks: parity 0 offsets 0, +1 (rows wl + 1, wl + 2), parity 1
                        // offsets -1, 0 (rows wl, wl + 1)
                        static_assert(CW == 16, "16 output channels per thread");
                        float a0[16], a1[16], b0[16], b1[16];
                        tmem_ld16x3(base + (unsigned)c, base + (unsigned)(NT + c), base + (unsigned)(2 * NT + c), a0,
                                    a1, b0);
                        tmem_ld16(base + (unsigned)(3 * NT + c), b1);
                        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                        __syncwarp();
                        if (lane == 0)
                            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(acce(ab)) : "memory");
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            b0[j] += __shfl_down_sync(0xffffffffu, a0[j], 1) + __shfl_down_sync(0xffffffffu, a1[j], 2) +
                                     __shfl_down_sync(0xffffffffu, b1[j], 1);
                        if (out_in && n < Nn) {
                            const long long v = (((long long)b * D + d_begin + i) * H + hl) * W + wc;
                            dwalk_store<16>(g, b0, nullptr, 0, out_bf16, out_f32, Nn, n, b, d_begin + i, hl, wc, v);
                        }
                    } else if constexpr (MODE == 2) {
                        float e0[CW], e1[CW], e2[CW], o0[CW], o1[CW], o2[CW];
                        tmem_ld8x3(base + (unsigned)c, base + (unsigned)(NT + c), base + (unsigned)(2 * NT + c), e0,
                                   e1, e2);
                        tmem_ld8x3(base + 64u + (unsigned)c, base + 64u + (unsigned)(NT + c),
                                   base + 64u + (unsigned)(2 * NT + c), o0, o1, o2);
                        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                        __syncwarp();
                        if (lane == 0)
                            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(acce(ab)) : "memory");
                        // pair P = m & 15 gives columns w0 + 2P and w0 + 2P + 1 (w0: first output)
#pragma unroll
                        for (int j = 0; j < CW; ++j) {
                            const float ne2 = __shfl_down_sync(0xffffffffu, e2[j], 1);
                            const float ne1 = __shfl_down_sync(0xffffffffu, e1[j], 1);
                            const float no2 = __shfl_down_sync(0xffffffffu, o2[j], 1);
                            e0[j] = e0[j] + o1[j] + ne2;
                            o0[j] = o0[j] + ne1 + no2;
                        }
                        const int wa = w0 + 2 * wl;
                        if (wl < 15 && hl < H && n < Nn) {
                            const long long v = (((long long)b * D + d_begin + i) * H + hl) * W + wa;
                            if (wa >= 0 && wa < W)
                                dwalk_store<CW>(g, e0, bias ? sBias + c : nullptr, relu, out_bf16, out_f32, Nn, n, b,
                                                d_begin + i, hl, wa, v);
                            if (wa + 1 < W)
                                dwalk_store<CW>(g, o0, bias ? sBias + c : nullptr, relu, out_bf16, out_f32, Nn, n, b,
                                                d_begin + i, hl, wa + 1, v + 1);
                        }
                    } else if constexpr (MODE == 0) {
                        float a0[CW], a1[CW], a2[CW];
                        if constexpr (CW == 16)
                            tmem_ld16x3(base + (unsigned)c, base + (unsigned)(NT + c), base + (unsigned)(2 * NT + c),
                                        a0, a1, a2);
                        else
                            tmem_ld8x3(base + (unsigned)c, base + (unsigned)(NT + c), base + (unsigned)(2 * NT + c),
                                       a0, a1, a2);
                        // the accumulator is free as soon as it is in registers
                        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                        __syncwarp();
                        if (lane == 0)
                            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(acce(ab)) : "memory");
#pragma unroll
                        for (int j = 0; j < CW; ++j)
                            a0[j] += __shfl_down_sync(0xffffffffu, a1[j], 1) + __shfl_down_sync(0xffffffffu, a2[j], 2);
                        if (out_in && n < Nn) {
                            const long long v = (((long long)b * D + d_begin + i) * H + hl) * W + wc;
                            dwalk_store<CW>(g, a0, bias ? sBias + c : nullptr, relu, out_bf16, out_f32, Nn, n, b,
                                            d_begin + i, hl, wc, v);
                        }
                    } else {
                        // blocks (pw, sw') = (0, 0), (0, 1), (1, 0), (1, 1): output column
                        // pw of coarse column wl adds blocks (pw, 0) of row wl + pw and
                        // (pw, 1) of row wl + pw + 1
                        float a0[CW], a1[CW], a2[CW], a3[CW];
                        if constexpr (CW == 16) {
                            tmem_ld16x3(base + (unsigned)c, base + (unsigned)(NT + c), base + (unsigned)(2 * NT + c),
                                        a0, a1, a2);
                            tmem_ld16(base + (unsigned)(3 * NT + c), a3);
                        } else {
                            tmem_ld8x3(base + (unsigned)c, base + (unsigned)(NT + c), base + (unsigned)(2 * NT + c),
                                       a0, a1, a2);
                            tmem_ld8(base + (unsigned)(3 * NT + c), a3);
                        }
                        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                        __syncwarp();
                        if (lane == 0)
                            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(acce(ab)) : "memory");
#pragma unroll
                        for (int j = 0; j < CW; ++j) {
                            const float b1 = __shfl_down_sync(0xffffffffu, a1[j], 1);
                            const float b2 = __shfl_down_sync(0xffffffffu, a2[j], 1);
                            const float b3 = __shfl_down_sync(0xffffffffu, a3[j], 2);
                            a0[j] += b1;
                            a2[j] = b2 + b3;
                        }
                        if (out_in && n < Nn) {
                            const int pd = u >> 1, ph = u & 1;
                            const int Do = 2 * D, Ho = 2 * H, Wo = 2 * W;
                            const int od = 2 * (d_begin + i) + pd, oh = 2 * hl + ph, ow = 2 * wc;
                            const long long v = (((long long)b * Do + od) * Ho + oh) * Wo + ow;
                            dwalk_store<CW>(g, a0, bias ? sBias + c : nullptr, relu, out_bf16, out_f32, Nn, n, b, od,
                                            oh, ow, v);
                            dwalk_store<CW>(g, a2, bias ? sBias + c : nullptr, relu, out_bf16, out_f32, Nn, n, b, od,
                                            oh, ow + 1, v + 1);
                        }
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0 && *abort_v) atomicExch(&g_tc_status, (int)FDC_ERR_TIMEOUT);
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kCols));
    }
}

// Collapsed weights of the data gradient of the upsampling convolution (MODE 3
// above): wt[ci][t][co], t = (((((qd qh qw) idx_d) idx_h) idx_w), the sum in FP32
// (rounded once to BF16) of w[co][kd][kh][kw][ci] over the taps of each axis
// with (q + k - 1) >> 1 = q - 1 + s', s' = 1 - idx (the collapse of the forward
// form, transposed).
__global__ void conv3_collapse_up_t_kernel(const __nv_bfloat16 *w, __nv_bfloat16 *wt, int co_n, int ci_n) {
    const long long n = (long long)co_n * 64 * ci_n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int co = (int)(i % co_n);
        const int t = (int)((i / co_n) % 64);
        const int ci = (int)(i / ((long long)co_n * 64));
        const int qd = (t >> 5) & 1, qh = (t >> 4) & 1, qw = (t >> 3) & 1;
        const int sd = 1 - ((t >> 2) & 1), sh = 1 - ((t >> 1) & 1), sw = 1 - (t & 1);
        float acc = 0.f;
        for (int kd = 0; kd < 3; ++kd) {
            if (((qd + kd - 1) >> 1) != qd - 1 + sd) continue;
            for (int kh = 0; kh < 3; ++kh) {
                if (((qh + kh - 1) >> 1) != qh - 1 + sh) continue;
                for (int kw = 0; kw < 3; ++kw) {
                    if (((qw + kw - 1) >> 1) != qw - 1 + sw) continue;
                    acc += __bfloat162float(w[((long long)co * 27 + (kd * 3 + kh) * 3 + kw) * ci_n + ci]);
                }
            }
        }
        wt[i] = __float2bfloat16_rn(acc);
    }
}

// Collapsed weights of the upsampling convolution (MODE 1 above):
// wc[co][pd ph][sd' sh'][pw sw'][ci] = sum of w[co][kd][kh][kw][ci] over the
// taps k of each axis with (p + k - 1) >> 1 = p - 1 + s', summed in FP32 and
// rounded once to BF16.
__global__ void conv3_collapse_up_kernel(const __nv_bfloat16 *w, __nv_bfloat16 *wc, int co_n, int ci_n) {
    const long long n = (long long)co_n * 64 * ci_n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(i % ci_n);
        const int t = (int)((i / ci_n) % 64);
        const int co = (int)(i / ((long long)ci_n * 64));
        // t = ((pd ph) * 4 + (sd' sh')) * 4 + (pw sw')
        const int pd = (t >> 5) & 1, ph = (t >> 4) & 1, sd = (t >> 3) & 1, sh = (t >> 2) & 1, pw = (t >> 1) & 1,
                  sw = t & 1;
        float acc = 0.f;
        for (int kd = 0; kd < 3; ++kd) {
            if (((pd + kd - 1) >> 1) != pd - 1 + sd) continue;
            for (int kh = 0; kh < 3; ++kh) {
                if (((ph + kh - 1) >> 1) != ph - 1 + sh) continue;
                for (int kw = 0; kw < 3; ++kw) {
                    if (((pw + kw - 1) >> 1) != pw - 1 + sw) continue;
                    acc += __bfloat162float(w[((long long)co * 27 + (kd * 3 + kh) * 3 + kw) * ci_n + ci]);
                }
            }
        }
        wc[i] = __float2bfloat16_rn(acc);
    }
}

// ---- weight gradient on the tcgen05 tensor cores, voxels as the reduction axis
//   dW[co][kd][kh][kw][ci] += sum over output voxels o of dy[o][co] * x[o + (kd, kh, kw) - 1][ci]
// (3^3, stride 1, padding 1).  K runs over (output plane d, output row h,
// input column wx); with the output column wo = wx + 1 - kw and kw' = 2 - kw,
//   D_kd[(kh, ci)][(kw', co)] += sum_k x[d + kd - 1][h + kh - 1][wx][ci] * dy[d][h][wx - 1 + kw'][co]
// is one MMA per kd for 16 consecutive planes d: M = 4 kh slots (the fourth
// discarded) x 8 CG input channels, N = 3 kw' x 16 output channels, K = 16.
// Both operands are MN-major (8 channels contiguous; the eight K rows of a
// core matrix are eight consecutive planes, 16 bytes apart): the input tile is
// stored [wx][h][channel group][d] and the gradient tile [h][wo][channel
// group][d], so every (kh, group) of A and every (kw', group) of B lies at one
// uniform stride from the first and the taps cost no copies.
// A CTA walks chunks of HT rows x WT columns x 16 planes (grid-stride),
// staging chunk i + 1 with cp.async while the MMAs of chunk i run (two
// buffers); the three accumulators (M x 48 FP32) stay in TMEM until its last
// chunk, are then laid out [co][tap][ci] in shared memory and added to dw
// with 16-byte vector reductions.  With db, the CTAs of the first input-channel
// slice also sum dy over their chunks into the bias gradient.  Every wait is
// bounded (FDC_ERR_TIMEOUT in g_tc_status on expiry).
constexpr int kWtDt = 16;          // output planes per chunk: one K run
constexpr int kWtThreads = 256;    // eight warps: staging in parallel, two CTAs per SM
constexpr int kWtDD = kWtDt + 2;   // input planes staged per chunk

template <int CG, int HT, int WT>
struct WgTc {
    static constexpr int HH = HT + 2, WO = WT + 2, CGO = 2, NCO = 16;
    static constexpr int M = 32 * CG, N = 24 * CGO;
    static constexpr int XBytes = WT * HH * CG * kWtDD * 16;
    static constexpr int YBytes = HT * WO * CGO * kWtDt * 16;
    static constexpr int BufBytes = XBytes + YBytes;
    static constexpr int Smem = 2 * BufBytes;
    static constexpr unsigned Cols = 3 * N <= 128 ? 128u : 256u;
    static constexpr int RedFloats = NCO * 27 * CG * 8;  // the CTA's dW block, [co][tap][ci]
    // A's discarded fourth kh slot of the last column reads past the input
    // tile, into the gradient tile that follows it
    static_assert(XBytes % 128 == 0 && BufBytes % 128 == 0, "128-byte aligned tiles");
    static_assert(YBytes >= CG * kWtDD * 16 + 512, "A's overrun stays in the buffer");
    static_assert(RedFloats * 4 <= Smem, "reduction tile fits the buffers");
};

__host__ __device__ constexpr unsigned umma_idesc_mn(int M, int N) {
    return umma_idesc(M, N) | (1u << 15) | (1u << 16);  // A and B MN-major
}

__device__ __forceinline__ void red_add_v4(float *p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

template <int CG, int HT, int WT>
__global__ void __launch_bounds__(kWtThreads) conv3_wgrad_tc_kernel(const Conv3dArgs g, const __nv_bfloat16 *x,
                                                             const __nv_bfloat16 *dy, float *dw, float *db, int ca,
                                                             int up_a, const __nv_bfloat16 *xb, int vec) {
    using P = WgTc<CG, HT, WT>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ unsigned tmem_slot;
    __shared__ float sBias[kWtThreads / 32][P::NCO];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int D = g.in_d, H = g.in_h, W = g.in_w, Ci = g.c_in, Co = g.c_out;
    const int co0 = blockIdx.y * P::NCO, ci0 = blockIdx.z * (8 * CG);
    const int cb = Ci - ca;
    const int Da = up_a ? D / 2 : D, Ha = up_a ? H / 2 : H, Wa = up_a ? W / 2 : W;
    const int tw = (W + WT - 1) / WT, th = (H + HT - 1) / HT, td = (D + kWtDt - 1) / kWtDt;
    const int n_chunks = g.batch * td * th * tw;  // the launcher checks that it fits
    const bool do_bias = db != nullptr && blockIdx.z == 0;
    const unsigned mb0 = smem_u32(&mbar[0]), mb1 = smem_u32(&mbar[1]);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb1));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(P::Cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const unsigned tmem = tmem_slot;

    // stage chunk ch into buf: input tile X[c][hh][cg][dd] (index order cg, c,
    // hh, dd: consecutive threads read consecutive 16-byte pieces of a row) and
    // gradient tile Y[r][wo][cgo][dd]; zero outside the grid
    // Input tile: each thread keeps one (column c, channel group cg) pair and
    // walks the (hh, dd) rows of it, so its source tensor, channel offset and
    // column are fixed (consecutive threads: consecutive 16-byte pieces of a
    // voxel row).  Gradient tile: index order cgo, wo, r, dd.
    constexpr int kPairs = CG * WT, kStep = kWtThreads / kPairs;
    static_assert(kWtThreads % kPairs == 0, "whole column pairs per pass");
    const int xcg = tid % CG, xc = (tid / CG) % WT, xrow0 = tid / kPairs;
    const int xch = ci0 + xcg * 8;
    const bool xfromb = xch >= ca;
    const __nv_bfloat16 *xsrc = xfromb ? xb : x;
    const int xC = xfromb ? cb : ca, xoff = xfromb ? xch - ca : xch, xup = xfromb ? 0 : up_a;
    const int xHs = xup ? Ha : H, xWs = xup ? Wa : W;
    const long long xplane = (long long)(xup ? Da : D) * xHs * xWs;
    const unsigned xdst0 = (unsigned)(((xc * P::HH) * CG + xcg) * kWtDD * 16);
    auto stage = [&](int ch, unsigned char *buf) {
        int t = ch;
        const int cw = t % tw;
        t /= tw;
        const int chh = t % th;
        t /= th;
        const int cd = t % td, b = t / td;
        const int d0 = cd * kWtDt, h0 = chh * HT, w0 = cw * WT;
        {
            const int w = w0 + xc;
            const bool w_in = w < W;
            const __nv_bfloat16 *base = xsrc + ((long long)b * xplane + (w >> xup)) * xC + xoff;
            for (int r = xrow0; r < P::HH * kWtDD; r += kStep) {
                const int hh = r / kWtDD, dd = r - hh * kWtDD;
                const int d = d0 - 1 + dd, h = h0 - 1 + hh;
                const bool in = w_in && (unsigned)d < (unsigned)D && (unsigned)h < (unsigned)H;
                const __nv_bfloat16 *p = in ? base + (long long)((d >> xup) * xHs + (h >> xup)) * xWs * xC : x;
                cp_async16(buf + xdst0 + (hh * CG * kWtDD + dd) * 16, p, in);
            }
        }
        unsigned char *yb = buf + P::XBytes;
        const __nv_bfloat16 *dyb = dy + (long long)b * D * H * W * Co + co0;
        for (int i = tid; i < HT * P::WO * P::CGO * kWtDt; i += kWtThreads) {
            const int cgo = i % P::CGO;
            int q = i / P::CGO;
            const int wo = q % P::WO;
            q /= P::WO;
            const int r = q % HT, dd = q / HT;
            const int d = d0 + dd, h = h0 + r, w = w0 - 1 + wo;
            const bool in = d < D && h < H && (unsigned)w < (unsigned)W;
            const __nv_bfloat16 *p = in ? dyb + ((long long)(d * H + h) * W + w) * Co + cgo * 8 : dy;
            cp_async16(yb + (((r * P::WO + wo) * P::CGO + cgo) * kWtDt + dd) * 16, p, in);
        }
    };
    float bsum[P::NCO];
#pragma unroll
    for (int j = 0; j < P::NCO; ++j) bsum[j] = 0.f;
    bool ok = true;
    int it = 0;
    int ch = blockIdx.x;
    if (ch < n_chunks) stage(ch, smem);
    cp_async_commit();
    for (; ch < n_chunks; ch += gridDim.x, ++it) {
        const int p = it & 1;
        unsigned char *buf = smem + p * P::BufBytes;
        cp_async_wait<0>();
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        // also agrees on the outcome of the previous iteration's bounded wait
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            constexpr unsigned idesc = umma_idesc_mn(P::M, P::N);
            // LBO: 128 bytes between K groups (8 planes); SBO: between M (N) groups
            const unsigned long long ad0 = umma_desc(smem_u32(buf), 128, kWtDD * 16);
            const unsigned long long bd0 = umma_desc(smem_u32(buf + P::XBytes), 128, kWtDt * 16);
#pragma unroll 1
            for (int r = 0; r < HT; ++r)
#pragma unroll 1
                for (int c = 0; c < WT; ++c) {
                    const unsigned long long bd = bd0 + (unsigned long long)((((r * P::WO + c) * P::CGO) * kWtDt));
                    const unsigned long long ad = ad0 + (unsigned long long)(((c * P::HH + r) * CG) * kWtDD);
                    const int acc = (it > 0 || r > 0 || c > 0) ? 1 : 0;
#pragma unroll
                    for (int kd = 0; kd < 3; ++kd)
                        umma_bf16(tmem + (unsigned)(kd * P::N), ad + (unsigned long long)kd, bd, idesc, acc);
                }
            umma_commit(p ? mb1 : mb0);
        }
        if (do_bias) {  // the chunk's own columns wo = 1 .. WT of the gradient tile
            const unsigned char *yb = buf + P::XBytes;
            for (int i = tid; i < HT * WT * kWtDt; i += kWtThreads) {
                const int dd = i % kWtDt, q = i / kWtDt;
                const int c = q % WT, r = q / WT;
#pragma unroll
                for (int cgo = 0; cgo < P::CGO; ++cgo) {
                    const uint4 v = *(const uint4 *)(yb + (((r * P::WO + c + 1) * P::CGO + cgo) * kWtDt + dd) * 16);
                    const __nv_bfloat162 *h2 = (const __nv_bfloat162 *)&v;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float2 f = __bfloat1622float2(h2[j]);
                        bsum[cgo * 8 + 2 * j] += f.x;
                        bsum[cgo * 8 + 2 * j + 1] += f.y;
                    }
                }
            }
        }
        // the other buffer is free once the previous chunk's MMAs are done
        if (it >= 1) ok = mbar_wait_bounded(p ? mb0 : mb1, ((it - 1) >> 1) & 1);
        const int nx = ch + (int)gridDim.x;
        if (ok && nx < n_chunks) stage(nx, smem + (p ^ 1) * P::BufBytes);
        cp_async_commit();
    }
    // the last chunk's MMAs complete after all earlier ones
    if (ok && it >= 1) ok = mbar_wait_bounded(((it - 1) & 1) ? mb1 : mb0, ((it - 1) >> 1) & 1);
    cp_async_wait<0>();
    ok = __syncthreads_and(ok);
    if (ok && it >= 1) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        // accumulator row of this thread (warp w reads the lanes of quadrant
        // w % 4): M = 128, the quadrant's rows; M = 64, rows 16 q .. 16 q + 15 in
        // lanes 0-15 of quadrant q.  Warps w and w + 4 take alternate 16-column blocks.
        const int quad = warp & 3, half = warp >> 2;
        const int m = P::M == 128 ? quad * 32 + lane : quad * 16 + lane;
        const bool row_ok = P::M == 128 || lane < 16;
        const int j = m >> 3, e = m & 7;
        const int kh = j / CG, cil = (j % CG) * 8 + e;
        const bool valid = row_ok && kh < 3;
        float *red = (float *)smem;  // [co][tap][ci] of this CTA; the buffers are idle now
#pragma unroll 1
        for (int blk = half; blk < 3 * (P::N / 16); blk += 2) {
            const int kd = blk / (P::N / 16), c16 = (blk % (P::N / 16)) * 16;
            {
                float v[16];
                tmem_ld16(tmem + ((unsigned)(quad * 32) << 16) + (unsigned)(kd * P::N + c16), v);
                if (valid)
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) {
                        const int n = c16 + jj, jn = n >> 3;
                        const int co = (jn % P::CGO) * 8 + (n & 7), kw = 2 - jn / P::CGO;
                        red[(co * 27 + (kd * 3 + kh) * 3 + kw) * (CG * 8) + cil] = v[jj];
                    }
            }
        }
        __syncthreads();
        // 16-byte pieces along ci: dw[(co0 + co) * 27 + tap][ci0 ..]
        constexpr int pieces = P::RedFloats / 4;
        for (int i = tid; i < pieces; i += kWtThreads) {
            const int f = i * 4;
            const int cil4 = f % (CG * 8), rest = f / (CG * 8);  // rest = co * 27 + tap
            const int co = rest / 27, tap = rest % 27;
            const float4 q = *(const float4 *)(red + f);
            float *dst = dw + ((long long)(co0 + co) * 27 + tap) * Ci + ci0 + cil4;
            if (vec) {
                red_add_v4(dst, q.x, q.y, q.z, q.w);
            } else {  // dw not 16-byte aligned
                atomicAdd(dst, q.x);
                atomicAdd(dst + 1, q.y);
                atomicAdd(dst + 2, q.z);
                atomicAdd(dst + 3, q.w);
            }
        }
        if (do_bias) {
#pragma unroll
            for (int jb = 0; jb < P::NCO; ++jb) {
                float v = bsum[jb];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) sBias[warp][jb] = v;
            }
            __syncthreads();
            if (tid < P::NCO) {
                float v = 0.f;
#pragma unroll
                for (int w = 0; w < kWtThreads / 32; ++w) v += sBias[w][tid];
                atomicAdd(db + co0 + tid, v);
            }
        }
    }
    if (!ok && tid == 0) atomicExch(&g_tc_status, (int)FDC_ERR_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(P::Cols));
    }
}

// ---- 2^3 stride-2 convolutions (the down-convolutions) on tcgen05.
// Output voxel v = (d, h, w) reads the 2 x 2 x 2 input block at (2d, 2h, 2w):
// tap t = (td * 2 + th) * 2 + tw, weights [co][t][ci].  Every input voxel
// belongs to exactly one block (the output grid is the input halved), so no
// tile needs a halo.
constexpr int kS2Vox = 128;      // output voxels per tile or K chunk
constexpr int kS2Threads = 256;

// Weight gradient dW[co][t][ci] += sum over v of dy[v][co] * x[2v + t][ci]:
// M = (tap, channel group) of a 16-channel input slice = 128 rows, N = Co
// (NCO), K = output voxels, 128 per chunk.  Both operands MN-major: A [tap][group][v][8 ch]
// (M groups 2048 bytes apart), B [co group][v][8 ch].  Chunks are staged with
// cp.async into two buffers (chunk i + 1 while chunk i's eight MMAs run), the
// accumulator stays in TMEM until the CTA's last chunk and is added to dw with
// 16-byte vector reductions; the CTAs of the first slice also sum dy into db.
template <int NCO>
__global__ void __launch_bounds__(kS2Threads) conv_s2_wgrad_tc_kernel(const Conv3dArgs g, const __nv_bfloat16 *x,
                                                                      const __nv_bfloat16 *dy, float *dw, float *db,
                                                                      int vec) {
    constexpr int CGO = NCO / 8;
    constexpr int ABytes = 16 * kS2Vox * 16, BBytes = CGO * kS2Vox * 16, Buf = ABytes + BBytes;
    constexpr unsigned Cols = NCO;
    static_assert(NCO * 8 * 16 * 4 <= 2 * Buf, "reduction tile fits the buffers");
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ unsigned tmem_slot;
    __shared__ float sb[NCO];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int D = g.in_d, H = g.in_h, W = g.in_w, Ci = g.c_in;
    const int D2 = g.out_d, H2 = g.out_h, W2 = g.out_w;
    const int ci0 = blockIdx.z * 16;
    const long long V = (long long)g.batch * D2 * H2 * W2;
    const int n_chunks = (int)((V + kS2Vox - 1) / kS2Vox);
    const bool do_bias = db != nullptr && blockIdx.z == 0;
    const unsigned mb0 = smem_u32(&mbar[0]), mb1 = smem_u32(&mbar[1]);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb1));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (tid < NCO) sb[tid] = 0.f;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(Cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const unsigned tmem = tmem_slot;
    // A: thread keeps q = (tw, group) and two voxels vA, vA + 64; 8 pieces per
    // chunk (tdh = k / 2).  B: thread keeps its co group and voxels stepping by
    // 256 / CGO.
    const int q = tid & 3, tw = q >> 1, cg = q & 1, vA = tid >> 2;
    const int bcgo = tid % CGO, bv0 = tid / CGO;
    constexpr int kBStep = kS2Threads / CGO;
    float bsum[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) bsum[j] = 0.f;
    auto voxel_base = [&](int v) -> const __nv_bfloat16 * {  // the launcher keeps V below 2^31
        const int w = v % W2;
        int t = v / W2;
        const int h = t % H2;
        t /= H2;
        const int d = t % D2, b = t / D2;
        return x + ((((long long)b * D + 2 * d) * H + 2 * h) * W + 2 * w + tw) * Ci + ci0 + cg * 8;
    };
    auto stage = [&](int ch, unsigned char *buf) {
        const long long v0 = (long long)ch * kS2Vox;
        const bool okA = v0 + vA < V, okB = v0 + vA + 64 < V;
        const __nv_bfloat16 *pa = okA ? voxel_base((int)(v0 + vA)) : x, *pb = okB ? voxel_base((int)(v0 + vA + 64)) : x;
        const long long sh = (long long)W * Ci, sd = (long long)H * W * Ci;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int tdh = k >> 1, vi = vA + (k & 1) * 64;
            const bool ok = (k & 1) ? okB : okA;
            const __nv_bfloat16 *p = (k & 1) ? pb : pa;
            const long long off = (tdh >> 1) * sd + (tdh & 1) * sh;
            const int tap = tdh * 2 + tw;
            cp_async16(buf + ((tap * 2 + cg) * kS2Vox + vi) * 16, ok ? p + off : x, ok);
        }
        unsigned char *bb = buf + ABytes;
#pragma unroll
        for (int vi = bv0; vi < kS2Vox; vi += kBStep) {
            const bool ok = v0 + vi < V;
            cp_async16(bb + (bcgo * kS2Vox + vi) * 16, ok ? dy + (v0 + vi) * g.c_out + bcgo * 8 : dy, ok);
        }
    };
    bool ok = true;
    int it = 0;
    int ch = blockIdx.x;
    if (ch < n_chunks) stage(ch, smem);
    cp_async_commit();
    for (; ch < n_chunks; ch += gridDim.x, ++it) {
        const int p = it & 1;
        unsigned char *buf = smem + p * Buf;
        cp_async_wait<0>();
        if (do_bias) {  // this thread's own staged dy pieces (zero past the end)
#pragma unroll
            for (int vi = bv0; vi < kS2Vox; vi += kBStep) {
                const uint4 u = *(const uint4 *)(buf + ABytes + (bcgo * kS2Vox + vi) * 16);
                const __nv_bfloat162 *h2 = (const __nv_bfloat162 *)&u;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float2 f = __bfloat1622float2(h2[j]);
                    bsum[2 * j] += f.x;
                    bsum[2 * j + 1] += f.y;
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            constexpr unsigned idesc = umma_idesc_mn(128, NCO);
            // LBO: 128 bytes between K groups (8 voxels); SBO: 2048 bytes between M (N) groups
            const unsigned long long ad0 = umma_desc(smem_u32(buf), 128, kS2Vox * 16);
            const unsigned long long bd0 = umma_desc(smem_u32(buf + ABytes), 128, kS2Vox * 16);
#pragma unroll
            for (int ks = 0; ks < kS2Vox / 16; ++ks)
                umma_bf16(tmem, ad0 + (unsigned long long)(ks * 16), bd0 + (unsigned long long)(ks * 16), idesc,
                          (it > 0 || ks > 0) ? 1 : 0);
            umma_commit(p ? mb1 : mb0);
        }
        if (it >= 1) ok = mbar_wait_bounded(p ? mb0 : mb1, ((it - 1) >> 1) & 1);
        const int nx = ch + (int)gridDim.x;
        if (ok && nx < n_chunks) stage(nx, smem + (p ^ 1) * Buf);
        cp_async_commit();
    }
    if (ok && it >= 1) ok = mbar_wait_bounded(((it - 1) & 1) ? mb1 : mb0, ((it - 1) >> 1) & 1);
    cp_async_wait<0>();
    ok = __syncthreads_and(ok);
    if (ok && it >= 1) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const int quad = warp & 3, half = warp >> 2;
        const int m = quad * 32 + lane;  // row (tap, group, channel)
        const int tap = m >> 4, cil = ((m >> 3) & 1) * 8 + (m & 7);
        float *red = (float *)smem;  // [co][tap][16 ci]
#pragma unroll 1
        for (int c16 = half * 16; c16 < NCO; c16 += 32) {
            float v[16];
            tmem_ld16(tmem + ((unsigned)(quad * 32) << 16) + (unsigned)c16, v);
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) red[((c16 + jj) * 8 + tap) * 16 + cil] = v[jj];
        }
        __syncthreads();
        for (int i = tid; i < NCO * 8 * 4; i += kS2Threads) {
            const int c4 = (i & 3) * 4, rest = i >> 2;  // rest = co * 8 + tap
            const float4 qv = *(const float4 *)(red + i * 4);
            float *dst = dw + (long long)rest * Ci + ci0 + c4;
            if (vec) {
                red_add_v4(dst, qv.x, qv.y, qv.z, qv.w);
            } else {
                atomicAdd(dst, qv.x);
                atomicAdd(dst + 1, qv.y);
                atomicAdd(dst + 2, qv.z);
                atomicAdd(dst + 3, qv.w);
            }
        }
        if (do_bias) {
#pragma unroll
            for (int j = 0; j < 8; ++j) atomicAdd(&sb[bcgo * 8 + j], bsum[j]);
            __syncthreads();
            if (tid < NCO) atomicAdd(db + tid, sb[tid]);
        }
    }
    if (!ok && tid == 0) atomicExch(&g_tc_status, (int)FDC_ERR_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(Cols));
    }
}

// Forward (MODE 0) and data gradient (MODE 1) of the 2^3 stride-2
// convolution: M = 128 output voxels per tile, K-major operands in the
// canonical no-swizzle layout (core matrices of 8 rows x 16 bytes), the
// weights resident in shared memory, A tiles double-buffered with cp.async
// and two TMEM accumulators, so that tile i's epilogue and tile i + 1's
// staging run while tile i's MMAs execute.
//   MODE 0: A[v][k] = x[2v + t][ci] with k = t Ci + ci (K = 8 Ci; the eight
//           2 x 2 x 2 block values of a voxel, two contiguous 2 Ci runs per
//           (td, th)), B[n = co][k] = w[co][t][ci]; epilogue bias, ReLU, y.
//   MODE 1: A[v][k = co] = dy[v][co] (K = Co), B[n][co] = w[co][t][ci] for the
//           N-tile's n = t Ci + ci (rows of w_t = [ci][t][co]); epilogue: the
//           16 columns of one tap are channels ci .. ci + 15 of input voxel
//           2v + t, masked by the ReLU derivative, plus the residual gradient
//           if given, and stored.
template <int MODE, int N, int K>
__global__ void __launch_bounds__(128) conv_s2_tc_kernel(const Conv3dArgs g, const __nv_bfloat16 *src,
                                                         const __nv_bfloat16 *wt, const float *bias,
                                                         __nv_bfloat16 *out_bf16, float *out_f32,
                                                         const __nv_bfloat16 *residual) {
    constexpr int ABytes = kS2Vox * K * 2, BBytes = N * K * 2;
    constexpr unsigned Cols = 2 * N;
    static_assert(Cols <= 512 && K % 16 == 0 && N % 16 == 0, "tile shape");
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ unsigned tmem_slot;
    unsigned char *sB = smem, *sA = smem + BBytes;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int D = g.in_d, H = g.in_h, W = g.in_w, Ci = g.c_in, Co = g.c_out;
    const int D2 = g.out_d, H2 = g.out_h, W2 = g.out_w;
    const int V = g.batch * D2 * H2 * W2;  // the launcher keeps it below 2^31
    const int n_tiles = (V + kS2Vox - 1) / kS2Vox;
    const int n0 = blockIdx.y * N;         // MODE 1: first column (t Ci + ci) of this N-tile
    const unsigned mb0 = smem_u32(&mbar[0]), mb1 = smem_u32(&mbar[1]);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb1));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(Cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const unsigned tmem = tmem_slot;
    // resident B: element (n, k) at ((k / 8) * (N / 8) + n / 8) * 128 + (n % 8) * 16 + (k % 8) * 2
    for (int i = tid; i < N * (K / 8); i += 128) {
        const int n = i % N, kg = i / N;
        const __nv_bfloat16 *p;
        if (MODE == 0) {
            p = wt + (long long)n * K + kg * 8;  // w[co][t Ci + ci]
        } else {
            const int col = n0 + n, t = col / Ci, ci = col % Ci;
            p = wt + ((long long)ci * 8 + t) * Co + kg * 8;  // w_t[ci][t][co]
        }
        cp_async16_ca(sB + ((kg * (N / 8) + n / 8) * 8 + (n % 8)) * 16, p, true);
    }
    // A tile of output voxels v0 .. v0 + 127: element (v, k) at
    // ((k / 8) * 16 + v / 8) * 128 + (v % 8) * 16 + (k % 8) * 2
    auto stage = [&](int tile, unsigned char *buf) {
        const int v0 = tile * kS2Vox;
        if (MODE == 0) {
            // per voxel and (td, th): 2 Ci contiguous values = 2 Ci / 8 pieces.
            // Piece i = tid + 128 m (m < PV) is piece i % PV of voxel i / PV: a
            // warp instruction covers 32 / PV whole voxels (contiguous runs),
            // and a warp's PV instructions cover 32 voxels, whose corner
            // addresses (2d, 2h, 2w) its lanes compute once, one voxel per
            // lane, and pass by shuffle.
            constexpr int PV = K / 8;  // pieces per voxel
            static_assert(PV <= 32 && 32 % PV == 0 && kS2Vox == 128, "staging map");
            constexpr int VPI = 32 / PV;  // voxels per warp instruction
            const int vl = (32 * warp) / PV + (lane / VPI) * (128 / PV) + lane % VPI;  // this lane's voxel
            long long corner = -1;  // element offset of the voxel's (2d, 2h, 2w) input, -1 past the end
            if (v0 + vl < V) {
                const int v = v0 + vl;
                const int w = v % W2;
                int t = v / W2;
                const int h = t % H2;
                t /= H2;
                const int d = t % D2, b = t / D2;
                corner = ((((long long)b * D + 2 * d) * H + 2 * h) * W + 2 * w) * Ci;
            }
#pragma unroll 4
            for (int m = 0; m < PV; ++m) {
                const int i = tid + 128 * m;
                const int j = i % PV, vi = i / PV;  // j = tdh * (PV / 4) + (piece within the run)
                const long long c = __shfl_sync(0xffffffffu, corner, m * VPI + lane / PV);
                const int tdh = j / (PV / 4), r = j % (PV / 4);
                const bool ok = c >= 0;
                const __nv_bfloat16 *p = ok ? src + c + ((long long)(tdh >> 1) * H + (tdh & 1)) * W * Ci + r * 8 : src;
                cp_async16(buf + ((j * 16 + vi / 8) * 8 + (vi % 8)) * 16, p, ok);
            }
        } else {
            constexpr int PV = K / 8;
            for (int i = tid; i < kS2Vox * PV; i += 128) {
                const int j = i % PV, vi = i / PV;
                const bool ok = v0 + vi < V;
                cp_async16(buf + ((j * 16 + vi / 8) * 8 + (vi % 8)) * 16,
                           ok ? src + (long long)(v0 + vi) * Co + j * 8 : src, ok);
            }
        }
    };
    // the MMAs of the tile in accumulator ab have completed (bounded wait;
    // the warp agrees on the outcome)
    auto acc_ready = [&](unsigned ab, unsigned ph) -> bool {
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(ab ? mb1 : mb0, ph))) return false;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        return true;
    };
    // epilogue of the tile in accumulator ab (after acc_ready): row m = this thread's voxel
    auto epilogue = [&](int tile, unsigned ab) {
        const int v = tile * kS2Vox + warp * 32 + lane;
        const bool in = v < V;
        int d = 0, h = 0, w = 0, b = 0;
        if (in) {
            w = v % W2;
            int t = v / W2;
            h = t % H2;
            t /= H2;
            d = t % D2;
            b = t / D2;
        }
        const unsigned base = tmem + ((unsigned)(warp * 32) << 16) + ab * N;
        if (MODE == 1 && in && (g.mask || residual)) {
            // the chunks below read the mask and residual rows one after the
            // other: ask L2 for all of them first, so that their DRAM latencies
            // overlap
#pragma unroll 1
            for (int c = 0; c < N; c += 16) {
                const int col = n0 + c, t = col / Ci, ci = col % Ci;
                const long long xv = (((long long)b * D + 2 * d + (t >> 2)) * H + 2 * h + ((t >> 1) & 1)) * W + 2 * w + (t & 1);
                if (g.mask) prefetch_l2((const __nv_bfloat16 *)g.mask + xv * Ci + ci);
                if (residual) prefetch_l2(residual + xv * Ci + ci);
            }
        }
#pragma unroll 1
        for (int c = 0; c < N; c += 16) {
            float a[16];
            tmem_ld16(base + (unsigned)c, a);
            if (!in) continue;
            if (MODE == 0) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    float x = a[j];
                    if (bias) x += __ldg(bias + c + j);
                    if (g.relu) x = fmaxf(x, 0.f);
                    a[j] = x;
                }
                if (out_f32) {
                    float4 *dst = (float4 *)(out_f32 + (long long)v * Co + c);
#pragma unroll
                    for (int j = 0; j < 4; ++j) dst[j] = make_float4(a[4 * j], a[4 * j + 1], a[4 * j + 2], a[4 * j + 3]);
                }
                if (out_bf16) {
                    uint4 qv[2];
                    unsigned *qq = (unsigned *)qv;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        __nv_bfloat162 p2 = __floats2bfloat162_rn(a[2 * j], a[2 * j + 1]);
                        qq[j] = *(unsigned *)&p2;
                    }
                    uint4 *dst = (uint4 *)(out_bf16 + (long long)v * Co + c);
                    dst[0] = qv[0];
                    dst[1] = qv[1];
                }
            } else {
                const int col = n0 + c, t = col / Ci, ci = col % Ci;
                const long long xv = (((long long)b * D + 2 * d + (t >> 2)) * H + 2 * h + ((t >> 1) & 1)) * W + 2 * w + (t & 1);
                if (g.mask) apply_relu_mask<16>(g.mask, xv, Ci, ci, a);
                if (residual) {  // a second gradient of the same activation, added before rounding
                    const uint4 *rp = (const uint4 *)(residual + xv * Ci + ci);
                    const uint4 rq[2] = {__ldg(rp), __ldg(rp + 1)};
                    const __nv_bfloat162 *r2 = (const __nv_bfloat162 *)rq;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float2 f = __bfloat1622float2(r2[j]);
                        a[2 * j] += f.x;
                        a[2 * j + 1] += f.y;
                    }
                }
                uint4 qv[2];
                unsigned *qq = (unsigned *)qv;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    __nv_bfloat162 p2 = __floats2bfloat162_rn(a[2 * j], a[2 * j + 1]);
                    qq[j] = *(unsigned *)&p2;
                }
                uint4 *dst = (uint4 *)(out_bf16 + xv * Ci + ci);
                dst[0] = qv[0];
                dst[1] = qv[1];
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    };
    bool ok = true;
    int it = 0;
    int tile = blockIdx.x;
    if (tile < n_tiles) stage(tile, sA);
    cp_async_commit();  // with the resident weights
    for (; tile < n_tiles; tile += gridDim.x, ++it) {
        const unsigned ab = it & 1u;
        unsigned char *buf = sA + ab * ABytes;
        cp_async_wait<0>();
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        // also agrees on the outcome of the previous epilogue's bounded wait
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            constexpr unsigned idesc = umma_idesc(128, N);
            // A: K groups 2048 bytes apart, 8-row groups 128; B: K groups N * 16 apart
            const unsigned long long ad0 = umma_desc(smem_u32(buf), kS2Vox * 16, 128);
            const unsigned long long bd0 = umma_desc(smem_u32(sB), N * 16, 128);
#pragma unroll
            for (int ks = 0; ks < K / 16; ++ks)
                umma_bf16(tmem + ab * N, ad0 + (unsigned long long)(ks * 2 * kS2Vox), bd0 + (unsigned long long)(ks * 2 * N),
                          idesc, ks > 0 ? 1 : 0);
            umma_commit(ab ? mb1 : mb0);
        }
        // once the previous tile's MMAs are done its A buffer takes the next
        // tile (the copies then run under that tile's epilogue)
        if (it > 0) ok = acc_ready(ab ^ 1u, ((it - 1) >> 1) & 1u);
        const int nx = tile + (int)gridDim.x;
        if (ok && nx < n_tiles) stage(nx, sA + (ab ^ 1u) * ABytes);
        cp_async_commit();
        if (it > 0 && ok) epilogue(tile - (int)gridDim.x, ab ^ 1u);
    }
    if (__syncthreads_and(ok) && it > 0) {
        ok = acc_ready((unsigned)(it - 1) & 1u, ((it - 1) >> 1) & 1u);
        if (ok) epilogue(blockIdx.x + (it - 1) * (int)gridDim.x, (unsigned)(it - 1) & 1u);
    } else {
        ok = ok && it == 0;
    }
    if (!ok && tid == 0) atomicExch(&g_tc_status, (int)FDC_ERR_TIMEOUT);
    cp_async_wait<0>();
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(Cols));
    }
}

// [ci][tap'][co] <- [co][tap][ci] with tap' the point reflection of tap
// (the data gradient of a stride-1 convolution is the forward convolution
// of dy with these weights)
__global__ void flip_transpose_kernel(const __nv_bfloat16 *w, __nv_bfloat16 *wf, int co_n, int k, int ci_n) {
    const int taps = k * k * k;
    const long long n = (long long)co_n * taps * ci_n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(i % ci_n);
        const long long q = i / ci_n;
        const int tap = (int)(q % taps), co = (int)(q / taps);
        wf[((long long)ci * taps + (taps - 1 - tap)) * co_n + co] = w[i];
    }
}

// Weight gradient: dW[co][tap][ci] += sum_v dy[v][co] * x[src(v, tap)][ci]
// over a chunk of output voxels v, as a GEMM with M = output channels,
// N = input channels and K = voxels; FP32 partial sums are added atomically.
constexpr int kWgVox = 16;        // voxels per K step
constexpr int kWgRowBytes = 144;  // 64 BF16 (128 B) padded to 144 B

// With db, the CTAs of tap 0 and the first input-channel tile also add the
// bias gradient of their output channels from the dy rows they stage.
__global__ void __launch_bounds__(128) conv_wgrad_kernel(const Conv3dArgs g, const __nv_bfloat16 *x,
                                                         const __nv_bfloat16 *dy, float *dw, float *db, int chunk) {
    __shared__ __align__(16) unsigned char sDy[2][kWgVox * kWgRowBytes];
    __shared__ __align__(16) unsigned char sX[2][kWgVox * kWgRowBytes];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int grp = lane >> 2, tig = lane & 3;
    const int taps = g.ksize * g.ksize * g.ksize;
    const int tap = blockIdx.y;
    const int kd = tap / (g.ksize * g.ksize), kh = (tap / g.ksize) % g.ksize, kw = tap % g.ksize;
    const int co_tiles = (g.c_out + 63) / 64;
    const int co0 = (blockIdx.x % co_tiles) * 64, ci0 = (blockIdx.x / co_tiles) * 64;
    const long long rows = (long long)g.batch * g.out_d * g.out_h * g.out_w;
    const long long v_begin = (long long)blockIdx.z * chunk;
    long long v_end = v_begin + chunk;
    if (v_end > rows) v_end = rows;
    const int ksteps = (int)((v_end - v_begin + kWgVox - 1) / kWgVox);

    // 16 voxels x 64 channels per operand: 128 chunks of 16 B each
    auto load_stage = [&](int buf, int ks) {
        const int vi = tid >> 3, part = tid & 7;  // voxel row, 8-channel part
        const long long v = v_begin + (long long)ks * kWgVox + vi;
        const bool vin = v < v_end;
        // dy row
        const int co = co0 + part * 8;
        const bool okd = vin && co < g.c_out;
        cp_async16(sDy[buf] + vi * kWgRowBytes + part * 16, okd ? dy + v * g.c_out + co : dy, okd);
        // x at the tap's source voxel
        long long sv = -1;
        if (vin) {
            const RowCoord rc = row_coord(v, rows, g.out_d, g.out_h, g.out_w);
            sv = src_voxel<0>(rc, kd, kh, kw, g);
        }
        const int ci = ci0 + part * 8;
        const bool okx = sv >= 0 && ci < g.c_in;
        cp_async16(sX[buf] + vi * kWgRowBytes + part * 16, okx ? x + sv * g.c_in + ci : x, okx);
    };
    auto ld16 = [](const unsigned char *base, int row, int col) -> unsigned {
        return (unsigned)*(const unsigned short *)(base + row * kWgRowBytes + col * 2);
    };

    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[j][k] = 0.f;
    const bool do_bias = db != nullptr && tap == 0 && ci0 == 0;
    float bsum[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // voxel row tid >> 3, channels (tid & 7) * 8 ..
    if (ksteps > 0) {
        load_stage(0, 0);
        cp_async_commit();
    }
    for (int ks = 0; ks < ksteps; ++ks) {
        const int buf = ks & 1;
        if (ks + 1 < ksteps) load_stage(buf ^ 1, ks + 1);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const unsigned char *Dy = sDy[buf];
        const unsigned char *X = sX[buf];
        if (do_bias) {  // this thread's staged 16-byte piece of dy (zero outside the chunk)
            const uint4 q = *(const uint4 *)(Dy + (tid >> 3) * kWgRowBytes + (tid & 7) * 16);
            const __nv_bfloat162 *h2 = (const __nv_bfloat162 *)&q;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 f = __bfloat1622float2(h2[j]);
                bsum[2 * j] += f.x;
                bsum[2 * j + 1] += f.y;
            }
        }
        // A[m = co][k = v]: warp rows co = warp * 16 + grp (+8); k = 2 tig (+1), (+8)
        const int m = warp * 16 + grp;
        const int k = tig * 2;
        const unsigned a0 = ld16(Dy, k, m) | (ld16(Dy, k + 1, m) << 16);
        const unsigned a1 = ld16(Dy, k, m + 8) | (ld16(Dy, k + 1, m + 8) << 16);
        const unsigned a2 = ld16(Dy, k + 8, m) | (ld16(Dy, k + 9, m) << 16);
        const unsigned a3 = ld16(Dy, k + 8, m + 8) | (ld16(Dy, k + 9, m + 8) << 16);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int n = nt * 8 + grp;
            const unsigned b0 = ld16(X, k, n) | (ld16(X, k + 1, n) << 16);
            const unsigned b1 = ld16(X, k + 8, n) | (ld16(X, k + 9, n) << 16);
            mma_bf16(acc[nt], a0, a1, a2, a3, b0, b1);
        }
        __syncthreads();
    }
    cp_async_wait<0>();
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int co = co0 + warp * 16 + grp + half * 8;
            const int ci = ci0 + nt * 8 + tig * 2;
            if (co >= g.c_out) continue;
            float *p = dw + ((long long)co * taps + tap) * g.c_in + ci;
            if (ci < g.c_in && acc[nt][half * 2] != 0.f) atomicAdd(p, acc[nt][half * 2]);
            if (ci + 1 < g.c_in && acc[nt][half * 2 + 1] != 0.f) atomicAdd(p + 1, acc[nt][half * 2 + 1]);
        }
    }
    if (do_bias) {  // the 16 voxel rows of each 8-channel part, reduced over the CTA
        __syncthreads();
        float *red = (float *)sX[0];  // 128 x 8 floats fit in the two x stages
#pragma unroll
        for (int j = 0; j < 8; ++j) red[tid * 8 + j] = bsum[j];
        __syncthreads();
        if (tid < 64) {
            const int part = tid >> 3, j = tid & 7, co = co0 + part * 8 + j;
            float t = 0.f;
            for (int vi = 0; vi < 16; ++vi) t += red[(vi * 8 + part) * 8 + j];
            if (co < g.c_out) atomicAdd(db + co, t);
        }
    }
}

// Several layers' data-gradient weights in one launch: entry e maps
// w[co][tap][ci] to wt[ci][tap'][co], tap' = taps - 1 - tap when flip (3^3
// stride-1 padding-1) else tap; element i of the batch belongs to the entry
// whose [start[e], start[e + 1]) holds it.
constexpr int kTrBatch = 32;
struct TransposeBatch {
    const __nv_bfloat16 *w[kTrBatch];
    __nv_bfloat16 *wt[kTrBatch];
    int co[kTrBatch], taps[kTrBatch], ci[kTrBatch], flip[kTrBatch];
    long long start[kTrBatch + 1];
    int n;
};

__global__ void transpose_batch_kernel(const TransposeBatch b) {
    const long long total = b.start[b.n];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        int e = 0;
        while (i >= b.start[e + 1]) ++e;
        const long long j = i - b.start[e];
        const int ci_n = b.ci[e], taps = b.taps[e], co_n = b.co[e];
        const int ci = (int)(j % ci_n);
        const long long q = j / ci_n;
        const int tap = (int)(q % taps), co = (int)(q / taps);
        const int tp = b.flip[e] ? taps - 1 - tap : tap;
        b.wt[e][((long long)ci * taps + tp) * co_n + co] = b.w[e][j];
    }
}

__global__ void transpose_weights_kernel(const __nv_bfloat16 *w, __nv_bfloat16 *wt, int co_n, int taps, int ci_n) {
    const long long n = (long long)co_n * taps * ci_n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(i % ci_n);
        const long long q = i / ci_n;
        const int tap = (int)(q % taps), co = (int)(q / taps);
        wt[((long long)ci * taps + tap) * co_n + co] = w[i];
    }
}

__global__ void relu_bwd_kernel(const __nv_bfloat16 *y, const __nv_bfloat16 *dy, __nv_bfloat16 *dx, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dx[i] = __bfloat162float(y[i]) > 0.f ? dy[i] : __float2bfloat16_rn(0.f);
}

// nearest x2 upsampling of [b][d][h][w][c] to [b][2d][2h][2w][c]
__global__ void upsample2_fwd_kernel(const __nv_bfloat16 *x, __nv_bfloat16 *y, int B, int D, int H, int W, int C) {
    const long long n = (long long)B * 8 * D * H * W * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        long long q = i / C;
        const int w = (int)(q % (2 * W)); q /= 2 * W;
        const int h = (int)(q % (2 * H)); q /= 2 * H;
        const int d = (int)(q % (2 * D));
        const int b = (int)(q / (2 * D));
        y[i] = x[((((long long)b * D + d / 2) * H + h / 2) * W + w / 2) * C + c];
    }
}

__global__ void upsample2_bwd_kernel(const __nv_bfloat16 *dy, __nv_bfloat16 *dx, int B, int D, int H, int W, int C) {
    const long long n = (long long)B * D * H * W * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        long long q = i / C;
        const int w = (int)(q % W); q /= W;
        const int h = (int)(q % H); q /= H;
        const int d = (int)(q % D);
        const int b = (int)(q / D);
        float s = 0.f;
        for (int k = 0; k < 8; ++k) {
            const int dd = 2 * d + (k >> 2), hh = 2 * h + ((k >> 1) & 1), ww = 2 * w + (k & 1);
            s += __bfloat162float(dy[((((long long)b * 2 * D + dd) * 2 * H + hh) * 2 * W + ww) * C + c]);
        }
        dx[i] = __float2bfloat16_rn(s);
    }
}

// out[r] = [a[r] | b[r]] along channels; split is the inverse (with da, db)
__global__ void concat_kernel(const __nv_bfloat16 *a, int Ca, const __nv_bfloat16 *b, int Cb, __nv_bfloat16 *out,
                              long long rows, int inverse) {
    const int C = Ca + Cb;
    const long long n = rows * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / C;
        const int c = (int)(i % C);
        if (!inverse) {
            out[i] = c < Ca ? a[r * Ca + c] : b[r * Cb + (c - Ca)];
        } else {
            if (c < Ca) ((__nv_bfloat16 *)a)[r * Ca + c] = out[i];
            else ((__nv_bfloat16 *)b)[r * Cb + (c - Ca)] = out[i];
        }
    }
}

// Mean squared error over rows of channel 0 of pred[rows][C] (FP32) against
// target[rows]; writes the BF16 gradient [rows][C] (zero outside channel 0)
// and adds the loss to *loss (per-block partial sums).
__global__ void mse_kernel(const float *pred, int C, const float *target, long long rows, float scale,
                           __nv_bfloat16 *grad, float *loss, int vec) {
    __shared__ float sm[256];
    float s = 0.f;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows; r += (long long)gridDim.x * blockDim.x) {
        const float e = pred[r * C] - target[r];
        s += e * e;
        if (grad) {
            if (vec) {  // whole 16-byte groups of the row (C % 8 == 0, aligned): channel 0, then zeros
                const __nv_bfloat16 g0 = __float2bfloat16_rn(2.f * e * scale);
                uint4 *row = (uint4 *)(grad + r * C);
                row[0] = make_uint4((unsigned)*(const unsigned short *)&g0, 0u, 0u, 0u);
                for (int k = 1; k < C / 8; ++k) row[k] = make_uint4(0u, 0u, 0u, 0u);
            } else {
                grad[r * C] = __float2bfloat16_rn(2.f * e * scale);
                for (int c = 1; c < C; ++c) grad[r * C + c] = __float2bfloat16_rn(0.f);
            }
        }
    }
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, sm[0] * scale);
}

// Adam (Kingma & Ba) on FP32 master weights; writes the BF16 copy.
__global__ void adam_kernel(float *p, const float *g, float *m, float *v, __nv_bfloat16 *p_bf16, long long n,
                            float lr, float b1, float b2, float eps, float bc1, float bc2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float upd = lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        const float pi = p[i] - upd;
        p[i] = pi;
        if (p_bf16) p_bf16[i] = __float2bfloat16_rn(pi);
    }
}

__global__ void f32_to_bf16_kernel(const float *x, __nv_bfloat16 *y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

__global__ void add_bf16_kernel(const __nv_bfloat16 *a, const __nv_bfloat16 *b, __nv_bfloat16 *out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16_rn(__bfloat162float(a[i]) + __bfloat162float(b[i]));
}

// Network input [n][16]: channel 0 = dose / dose_scale, channel 1 = density *
// density_scale, the rest zero; dose_in keeps channel 0 in FP32 and, with a
// high-history dose, target = dose_high / dose_scale - dose_in (the network
// predicts the correction to its input).
__global__ void prepare_kernel(const double *dose, const float *density, const double *dose_high, long long n,
                               double inv_scale, float density_scale, __nv_bfloat16 *x, float *dose_in,
                               float *target, const double *scale_dev) {
    // scale_dev: the dose scale in device memory (a non-positive scale counts as 1)
    if (scale_dev) inv_scale = 1.0 / (*scale_dev > 0.0 ? *scale_dev : 1.0);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = (float)(dose[i] * inv_scale);
        dose_in[i] = d;
        // the 32-byte row as two 16-byte stores: channels 0 and 1, then zeros
        const __nv_bfloat162 c01 = __floats2bfloat162_rn(d, density[i] * density_scale);
        uint4 q0 = make_uint4(*(const unsigned *)&c01, 0u, 0u, 0u);
        uint4 *row = (uint4 *)(x + i * 16);
        row[0] = q0;
        row[1] = make_uint4(0u, 0u, 0u, 0u);
        if (target) target[i] = (float)(dose_high[i] * inv_scale) - d;
    }
}

// Lateral symmetry of a field along +z: out[d][h][w] = in[d][h'][w'] with
// (h', w') the image of (h, w) under code (bit 0: mirror w, bit 1: mirror h,
// bit 2: exchange h and w; h == w when bit 2 is set).  One 32-byte row of 16
// bf16 channels per voxel of x, one FP32 value per voxel of t.
__global__ void dihedral_kernel(const uint4 *x, const float *t, int D, int H, int W, int code, uint4 *xo,
                                float *to) {
    const long long n = (long long)D * H * W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int w = (int)(i % W);
        const int h = (int)((i / W) % H);
        const long long d = i / ((long long)W * H);
        int hs = (code & 4) ? w : h, ws = (code & 4) ? h : w;
        if (code & 1) ws = W - 1 - ws;
        if (code & 2) hs = H - 1 - hs;
        const long long j = (d * H + hs) * W + ws;
        xo[2 * i] = x[2 * j];
        xo[2 * i + 1] = x[2 * j + 1];
        if (t) to[i] = t[j];
    }
}

__global__ void finish_kernel(const float *head, const float *dose_in, long long n, double scale, double *dose_out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = ((double)head[i * 16] + (double)dose_in[i]) * scale;
        dose_out[i] = v > 0.0 ? v : 0.0;
    }
}

// ---- head of the denoiser: output channel 0 of its 1^3 convolution, the only
// channel the loss and the denoised dose use: y = b[0] + sum_c w[c] x[c] over
// the 16 BF16 feature channels of a voxel (exact BF16 products, FP32 sum).
__device__ __forceinline__ void load_row16(const __nv_bfloat16 *__restrict__ x, long long i, float f[16]) {
    const uint4 *row = (const uint4 *)(x + i * 16);
    const uint4 q[2] = {row[0], row[1]};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const unsigned u[4] = {q[k].x, q[k].y, q[k].z, q[k].w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 v = __bfloat1622float2(*(const __nv_bfloat162 *)&u[j]);
            f[8 * k + 2 * j] = v.x;
            f[8 * k + 2 * j + 1] = v.y;
        }
    }
}

__device__ __forceinline__ float head_dot(const float w[16], const float f[16], float b0) {
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 16; ++c) s = fmaf(w[c], f[c], s);
    return s + b0;
}

// Inference: y (may be NULL) = the correction; dose_out (may be NULL) =
// max(0, (y + dose_in) * scale).
__global__ void head_kernel(const __nv_bfloat16 *__restrict__ x, const __nv_bfloat16 *__restrict__ w,
                            const float *__restrict__ b, long long n, const float *__restrict__ dose_in, double scale,
                            float *__restrict__ y, double *__restrict__ dose_out, const double *scale_dev) {
    if (scale_dev) scale = *scale_dev > 0.0 ? *scale_dev : 1.0;
    float wf[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) wf[c] = __bfloat162float(w[c]);
    const float b0 = b[0];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float f[16];
        load_row16(x, i, f);
        const float v = head_dot(wf, f, b0);
        if (y) y[i] = v;
        if (dose_out) {
            const double d = ((double)v + (double)dose_in[i]) * scale;
            dose_out[i] = d > 0.0 ? d : 0.0;
        }
    }
}

// Training: loss += mean over voxels of (y - target)^2; with g = 2 (y - target) / n,
// dx (may be NULL) = bf16(w[c] g) where x[c] > 0 (the ReLU derivative of the
// layer that produced x), else 0; dw[c] += sum g x[c] and db[0] += sum g
// (dw NULL: no weight gradient).  Block partial sums, one FP32 atomic per
// block and value.
__global__ void __launch_bounds__(256) head_loss_kernel(const __nv_bfloat16 *__restrict__ x,
                                                        const __nv_bfloat16 *__restrict__ w,
                                                        const float *__restrict__ b, const float *__restrict__ target,
                                                        long long n, float inv_n, float *loss,
                                                        __nv_bfloat16 *__restrict__ dx, float *dw, float *db) {
    __shared__ float part[8][18];
    float wf[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) wf[c] = __bfloat162float(w[c]);
    const float b0 = b[0];
    float acc[18];  // 0..15: weight gradient, 16: bias gradient, 17: squared error
#pragma unroll
    for (int k = 0; k < 18; ++k) acc[k] = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float f[16];
        load_row16(x, i, f);
        const float e = head_dot(wf, f, b0) - target[i];
        acc[17] = fmaf(e, e, acc[17]);
        const float g = 2.f * e * inv_n;
        if (dx) {
            unsigned u[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * j] > 0.f ? wf[2 * j] * g : 0.f,
                                                               f[2 * j + 1] > 0.f ? wf[2 * j + 1] * g : 0.f);
                u[j] = *(const unsigned *)&h;
            }
            uint4 *row = (uint4 *)(dx + i * 16);
            row[0] = make_uint4(u[0], u[1], u[2], u[3]);
            row[1] = make_uint4(u[4], u[5], u[6], u[7]);
        }
        if (dw) {
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[c] = fmaf(g, f[c], acc[c]);
            acc[16] += g;
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 18; ++k) {
        float v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) part[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 18) {
        float v = 0.f;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v += part[q][threadIdx.x];
        if (threadIdx.x == 17) atomicAdd(loss, v * inv_n);
        else if (dw && threadIdx.x == 16) atomicAdd(db, v);
        else if (dw) atomicAdd(dw + threadIdx.x, v);
    }
}

// ---- gamma index (Low et al. 1998), global dose difference
// gamma(v) = min over evaluated points u within the search radius of
// sqrt(|u - v|^2 / dta^2 + (eval(u) - ref(v))^2 / (dd * ref_max)^2),
// for reference voxels with ref(v) > threshold * ref_max.
__global__ void max_kernel(const double *x, long long n, unsigned long long *out) {
    __shared__ double sm[256];
    double m = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmax(m, x[i]);
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
        __syncthreads();
    }
    // non-negative doubles order like their bit patterns
    if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(sm[0]));
}

__global__ void gamma_kernel(const double *ref, const double *eval, int D, int H, int W, double sd, double sh,
                             double sw, double dd, double dta, double thr, int radius,
                             const unsigned long long *ref_max_bits, float *gamma, unsigned long long *counts) {
    const double ref_max = __longlong_as_double((long long)*ref_max_bits);
    const double dmax = dd * ref_max;
    const long long n = (long long)D * H * W;
    unsigned long long evaluated = 0, passed = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double r = ref[i];
        if (!(r > thr * ref_max)) {
            if (gamma) gamma[i] = -1.f;
            continue;
        }
        const int w = (int)(i % W), h = (int)((i / W) % H), d = (int)(i / ((long long)W * H));
        double best = 1e300;
        for (int a = -radius; a <= radius; ++a) {
            const int dz = d + a;
            if (dz < 0 || dz >= D) continue;
            for (int b = -radius; b <= radius; ++b) {
                const int hy = h + b;
                if (hy < 0 || hy >= H) continue;
                for (int c = -radius; c <= radius; ++c) {
                    const int wx = w + c;
                    if (wx < 0 || wx >= W) continue;
                    const double dist2 = (a * sd) * (a * sd) + (b * sh) * (b * sh) + (c * sw) * (c * sw);
                    const double de = eval[((long long)dz * H + hy) * W + wx] - r;
                    const double g2 = dist2 / (dta * dta) + de * de / (dmax * dmax);
                    best = fmin(best, g2);
                }
            }
        }
        const double gm = sqrt(best);
        if (gamma) gamma[i] = (float)gm;
        ++evaluated;
        if (gm <= 1.0) ++passed;
    }
    atomicAdd(counts, evaluated);
    atomicAdd(counts + 1, passed);
}

int grid_for(long long n, int threads = 256) {
    long long b = (n + threads - 1) / threads;
    if (b > 16384) b = 16384;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

// SM count and resident CTAs of one kernel at one shared-memory size, queried
// once per device (the caller holds one cache per kernel); the kernel's opt-in
// shared-memory limit is raised to the device maximum on first use.
struct OccCache {
    int v[16][16][3];  // [device][slot] = {smem, sms, per_sm}
    std::mutex mu;
};
template <typename K>
cudaError_t prepare_kernel_smem(OccCache &c, K kernel, int smem) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(c.mu);
    if (dev < 16)
        for (int i = 0; i < 16 && c.v[dev][i][0]; ++i)
            if (c.v[dev][i][0] == smem) return cudaSuccess;
    int maxopt = 0;
    e = cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, maxopt - 1024);
    // as much of the unified L1 / shared memory as shared memory as residency needs
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    if (dev < 16)
        for (int i = 0; i < 16; ++i)
            if (!c.v[dev][i][0]) {
                c.v[dev][i][0] = smem;
                break;
            }
    return cudaSuccess;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (the library links no driver stub).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// 5-D tensor map of a channels-last BF16 activation [batch][d][h][w][C] read
// in boxes of 16 channels x 16 w x 10 h x 1 d x 1 batch with the 32-byte
// swizzle (zero fill outside the grid); false when it cannot be made.
bool make_plane_map(CUtensorMap *m, const void *base, int C, int B, int D, int H, int W) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || !base || ((uintptr_t)base & 15u) || C % 16 || W < 16 || H < 10) return false;
    const cuuint64_t e = 2;  // bytes per element
    const cuuint64_t dims[5] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)B};
    const cuuint64_t strides[4] = {dims[0] * e, dims[0] * dims[1] * e, dims[0] * dims[1] * dims[2] * e,
                                   dims[0] * dims[1] * dims[2] * dims[3] * e};
    const cuuint32_t box[5] = {16, 16, 10, 1, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 5-D tensor map of a 16-channel channels-last BF16 activation read as pairs
// of neighbouring voxels (W even): 32 values x W/2 pairs x H x D x batch,
// boxes of 16 pairs x 10 h with the 64-byte swizzle; false when it cannot be made.
bool make_pair_map(CUtensorMap *m, const void *base, int B, int D, int H, int W) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || !base || ((uintptr_t)base & 15u) || W % 2 || W < 32 || H < 10) return false;
    const cuuint64_t dims[5] = {32, (cuuint64_t)W / 2, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)B};
    const cuuint64_t strides[4] = {64, 64 * dims[1], 64 * dims[1] * dims[2], 64 * dims[1] * dims[2] * dims[3]};
    const cuuint32_t box[5] = {32, 16, 10, 1, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// FP32 partial sums of a K-split convolution, per device: grown on demand,
// never while the stream is being captured into a graph, and a buffer once
// handed out is never freed (a captured graph may hold its address), so the
// buffers stay allocated until the process exits.
struct SplitScratch {
    float *p[16] = {};
    size_t n[16] = {};
    std::mutex mu;
};

cudaError_t split_scratch(size_t floats, cudaStream_t st, float **out) {
    static SplitScratch sc;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 16) return cudaErrorNotSupported;
    std::lock_guard<std::mutex> lock(sc.mu);
    if (sc.n[dev] < floats) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        e = cudaStreamIsCapturing(st, &cs);
        if (e != cudaSuccess) return e;
        if (cs != cudaStreamCaptureStatusNone) return cudaErrorNotSupported;  // no allocation inside a capture
        float *q = nullptr;
        e = cudaMalloc((void **)&q, floats * sizeof(float));
        if (e != cudaSuccess) return e;
        sc.p[dev] = q;  // the smaller buffer stays allocated (graphs may use it)
        sc.n[dev] = floats;
    }
    *out = sc.p[dev];
    return cudaSuccess;
}

// out[i] = act(bias[i % Nn] + sum over the splits of part[s][i]), in split order;
// with mask (a data gradient: the layer's forward input, the output's layout),
// zero where mask[i] is not positive.
__global__ void split_combine_kernel(const float *part, int splits, long long n, const float *bias, int Nn, int relu,
                                     const __nv_bfloat16 *mask, __nv_bfloat16 *out_bf16, float *out_f32) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n / 4; q += stride) {
        float4 a = ((const float4 *)part)[q];
        for (int sp = 1; sp < splits; ++sp) {
            const float4 b = ((const float4 *)(part + (long long)sp * n))[q];
            a.x += b.x;
            a.y += b.y;
            a.z += b.z;
            a.w += b.w;
        }
        float v[4] = {a.x, a.y, a.z, a.w};
        const int c0 = (int)((4 * q) % Nn);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (bias) v[j] += bias[c0 + j];
            if (relu) v[j] = fmaxf(v[j], 0.f);
        }
        if (mask) {
            const uint2 mq = ((const uint2 *)mask)[q];
            const unsigned short mh[4] = {(unsigned short)(mq.x & 0xffffu), (unsigned short)(mq.x >> 16),
                                          (unsigned short)(mq.y & 0xffffu), (unsigned short)(mq.y >> 16)};
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if ((short)mh[j] <= 0) v[j] = 0.f;  // sign bit set, or +0: not positive
        }
        if (out_f32) ((float4 *)out_f32)[q] = make_float4(v[0], v[1], v[2], v[3]);
        if (out_bf16) {
            const __nv_bfloat162 p0 = __floats2bfloat162_rn(v[0], v[1]), p1 = __floats2bfloat162_rn(v[2], v[3]);
            uint2 u;
            u.x = *(const unsigned *)&p0;
            u.y = *(const unsigned *)&p1;
            ((uint2 *)out_bf16)[q] = u;
        }
    }
}

// 5-D tensor map of a full-resolution channels-last BF16 tensor read by parity
// class: boxes of 16 channels x 16 w x 10 h taken every second voxel along w
// and h (element strides 2), 32-byte swizzle; false when it cannot be made.
bool make_parity_map(CUtensorMap *m, const void *base, int C, int B, int D, int H, int W) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || !base || ((uintptr_t)base & 15u) || C % 16 || W < 32 || H < 20) return false;
    const cuuint64_t e = 2;
    const cuuint64_t dims[5] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)B};
    const cuuint64_t strides[4] = {dims[0] * e, dims[0] * dims[1] * e, dims[0] * dims[1] * dims[2] * e,
                                   dims[0] * dims[1] * dims[2] * dims[3] * e};
    const cuuint32_t box[5] = {16, 32, 20, 1, 1};
    const cuuint32_t estr[5] = {1, 2, 2, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The TMA d-walking kernel.  MODE 0: an input read as stored (no upsampling;
// the split of a two-part input on a 16-channel boundary).  MODE 1: the
// sub-pixel form of the convolution of upsample2(src), src on the coarse grid
// with Cs channels, wt the collapsed weights.  MODE 3: the data gradient of
// that convolution on the coarse grid, src = dy at full resolution with Cs
// channels, wt the transposed collapsed weights, Nn = the coarse input's
// channels.  splits > 1: the Cs input
// channels are split into `splits` equal parts of at most 64 over
// blockIdx.z, each part's FP32 partial sums written to scratch, and one
// combine pass adds them in order with the bias, the ReLU and a data
// gradient's plain ReLU mask (g.mask with g.mask_ca = 0; no split output).
// cudaErrorNotSupported, launching nothing, when the shape has no
// instantiation or its tensor maps cannot be made.
cudaError_t launch_dwtma(int mode, const Conv3dArgs &g, const __nv_bfloat16 *src, const __nv_bfloat16 *wt,
                         const float *bias, __nv_bfloat16 *out_bf16, float *out_f32, int Cs, int Nn, int relu,
                         cudaStream_t st, int ca, const __nv_bfloat16 *src_b, int splits = 1) {
    if (splits < 1 || Cs % splits || (Cs / splits) % 16 || Cs / splits > 64 || Nn % 16 || ca % 16 ||
        (Cs - ca) % 16 || (ca < Cs && !src_b))
        return cudaErrorNotSupported;
    if ((mode == 1 || mode == 3) && (ca != Cs || g.in_d % 2 || g.in_h % 2 || g.in_w % 2))
        return cudaErrorNotSupported;
    if (splits > 1 && (g.mask_ca > 0 || g.out_b)) return cudaErrorNotSupported;
    // the walked (input) grid
    const int D = mode ? g.in_d / 2 : g.in_d, H = mode ? g.in_h / 2 : g.in_h, W = mode ? g.in_w / 2 : g.in_w;
    CUtensorMap tm_a, tm_b;
    // pair tiles when the input is two 16-channel tensors and w is even (measured at 128^3:
    // [16 | 16] -> 16 94 vs 118 us; for one 16-channel tensor the two CTAs per SM that their
    // accumulators leave were slower than four with plain tiles, 66 vs 62 us)
    if (mode == 0 && splits == 1 && FDC_DWT_PAIR && ca == 16 && Cs == 32 &&
        make_pair_map(&tm_a, src, g.batch, D, H, W) && make_pair_map(&tm_b, src_b, g.batch, D, H, W))
        mode = 2;
    if (mode == 3) {
        if (!make_parity_map(&tm_a, src, Cs, g.batch, g.in_d, g.in_h, g.in_w)) return cudaErrorNotSupported;
    } else if (mode != 2 && !make_plane_map(&tm_a, src, ca, g.batch, D, H, W)) {
        return cudaErrorNotSupported;
    }
    if (ca == Cs) {
        tm_b = tm_a;
    } else if (mode != 2 && !make_plane_map(&tm_b, src_b, Cs - ca, g.batch, D, H, W)) {
        return cudaErrorNotSupported;
    }
    int dev = 0, sms = 0, smem_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e != cudaSuccess) return e;
    const int Cp = Cs / splits;  // input channels per CTA
    const int S = Cp / 16;
    const int NT = ((mode == 0 || mode == 3) && Nn % 32 == 0) ? 32 : 16;
    const int NX = (mode == 1 ? 4 : (mode == 3 ? 2 : 3)) * NT, NU = mode == 1 ? 16 : (mode == 3 ? 32 : 9);
    const int wbytes = S * NU * 2 * NX * 16;
    const int plane = S * kDwPlaneSliceBytes * (mode == 2 ? 2 : (mode == 3 ? 4 : 1));
    // CTAs per SM: at most what TMEM allows (accumulator slots of 64 or 128 of
    // the 512 columns: two per CTA in MODE 0, one coarse plane's four units
    // in MODE 1), fewer when the ring would hold less than 5 planes (three in
    // use, two in flight) or, in MODE 1, 4; one CTA per SM takes a ring of 4
    int per_sm = mode != 0 ? 2 : (NT == 32 ? 2 : 4), R = 0;
    const int r_min = mode == 3 ? 6 : (mode != 0 ? 4 : 5);  // MODE 3: four planes in use, two in flight
    for (; per_sm > 1; --per_sm) {
        R = std::min(kDwtMaxRing, (smem_sm / per_sm - 3072 - wbytes - 1024) / plane);
        if (R >= r_min) break;
    }
    if (per_sm == 1) R = std::min(kDwtMaxRing, (smem_sm - 3072 - wbytes - 1024) / plane);
    if (R < (mode == 3 ? 6 : 4)) return cudaErrorNotSupported;
    const int NA = mode != 1 ? 2 : (per_sm == 2 ? 4 : 8);
    const int smem = wbytes + 1024 + R * plane;
    const int ntiles = (Nn + NT - 1) / NT;
    const long long planes =
        (long long)g.batch * ((H + 7) / 8) * (mode == 2 ? (W + 30) / 30 : (W + 13) / 14) * D;
    long long gx = std::max(1ll, (long long)sms * per_sm / (ntiles * splits));
    if (gx > planes) gx = planes;
    const dim3 grid((unsigned)gx, (unsigned)ntiles, (unsigned)splits);
    // split partial sums: [splits][output voxels][Nn] FP32
    const long long n_out = (long long)g.batch * (mode == 3 ? (long long)D * H * W : (long long)g.in_d * g.in_h * g.in_w) * Nn;
    float *part = nullptr;
    if (splits > 1) {
        e = split_scratch((size_t)n_out * splits, st, &part);
        if (e != cudaSuccess) return e;
    }
    Conv3dArgs gk = g;  // the split partials carry no mask: the combine pass applies it
    if (splits > 1) gk.mask = nullptr;
    const float *kb = splits > 1 ? nullptr : bias;
    __nv_bfloat16 *kob = splits > 1 ? nullptr : out_bf16;
    float *kof = splits > 1 ? part : out_f32;
    const int krelu = splits > 1 ? 0 : relu;
    if (mode == 3 && NT == 32) {
        static OccCache cache;
        e = prepare_kernel_smem(cache, conv3_dwtma_kernel<32, 8, 1, 3>, smem);
        if (e != cudaSuccess) return e;
        conv3_dwtma_kernel<32, 8, 1, 3><<<grid, 320, smem, st>>>(tm_a, tm_b, gk, wt, kb, kob, kof, Cp, Nn, krelu, ca,
                                                                  R, NA, Cs, n_out);
    } else if (mode == 3) {
        static OccCache cache;
        e = prepare_kernel_smem(cache, conv3_dwtma_kernel<16, 4, 2, 3>, smem);
        if (e != cudaSuccess) return e;
        conv3_dwtma_kernel<16, 4, 2, 3><<<grid, 192, smem, st>>>(tm_a, tm_b, gk, wt, kb, kob, kof, Cp, Nn, krelu, ca,
                                                                  R, NA, Cs, n_out);
    } else if (mode == 2) {
        static OccCache cache;
        e = prepare_kernel_smem(cache, conv3_dwtma_kernel<16, 8, 2, 2>, smem);
        if (e != cudaSuccess) return e;
        conv3_dwtma_kernel<16, 8, 2, 2><<<grid, 320, smem, st>>>(tm_a, tm_b, gk, wt, kb, kob, kof, Cp, Nn, krelu, ca,
                                                                  R, NA, Cs, n_out);
    } else if (mode == 1) {
        static OccCache cache;
        e = prepare_kernel_smem(cache, conv3_dwtma_kernel<16, 8, 2, 1>, smem);
        if (e != cudaSuccess) return e;
        conv3_dwtma_kernel<16, 8, 2, 1><<<grid, 320, smem, st>>>(tm_a, tm_b, gk, wt, kb, kob, kof, Cp, Nn, krelu, ca,
                                                                  R, NA, Cs, n_out);
    } else if (NT == 32) {
        static OccCache cache;
        e = prepare_kernel_smem(cache, conv3_dwtma_kernel<32, 8, 2, 0>, smem);
        if (e != cudaSuccess) return e;
        conv3_dwtma_kernel<32, 8, 2, 0><<<grid, 320, smem, st>>>(tm_a, tm_b, gk, wt, kb, kob, kof, Cp, Nn, krelu, ca,
                                                                  R, NA, Cs, n_out);
    } else if (per_sm >= 3) {
        static OccCache cache;
        e = prepare_kernel_smem(cache, conv3_dwtma_kernel<16, 4, 4, 0>, smem);
        if (e != cudaSuccess) return e;
        conv3_dwtma_kernel<16, 4, 4, 0><<<grid, 192, smem, st>>>(tm_a, tm_b, gk, wt, kb, kob, kof, Cp, Nn, krelu, ca,
                                                                  R, NA, Cs, n_out);
    } else {
        static OccCache cache;
        e = prepare_kernel_smem(cache, conv3_dwtma_kernel<16, 8, 2, 0>, smem);
        if (e != cudaSuccess) return e;
        conv3_dwtma_kernel<16, 8, 2, 0><<<grid, 320, smem, st>>>(tm_a, tm_b, gk, wt, kb, kob, kof, Cp, Nn, krelu, ca,
                                                                  R, NA, Cs, n_out);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess || splits == 1) return e;
    long long blocks = (n_out / 4 + 255) / 256;
    if (blocks > (long long)sms * 16) blocks = (long long)sms * 16;
    split_combine_kernel<<<(int)blocks, 256, 0, st>>>(part, splits, n_out, bias, Nn, relu,
                                                      (const __nv_bfloat16 *)g.mask, out_bf16, out_f32);
    return cudaGetLastError();
}

cudaError_t launch_conv_up(const Conv3dArgs &g, const void *xa, const void *w_up, const float *bias, void *out_bf16,
                           float *out_f32, int relu, cudaStream_t st) {
    // more than 64 input channels: K split into 32-channel parts (their collapsed weights fit)
    const int splits = g.c_in > 64 && FDC_DWT_KSPLIT ? g.c_in / 32 : 1;
    return launch_dwtma(1, g, (const __nv_bfloat16 *)xa, (const __nv_bfloat16 *)w_up, bias, (__nv_bfloat16 *)out_bf16,
                        out_f32, g.c_in, g.c_out, relu, st, g.c_in, nullptr, splits);
}

// the data gradient of the sub-pixel upsampling convolution: dy (full resolution,
// g.c_out channels) to dxa (coarse, g.c_in channels, masked by relu_mask = xa > 0)
cudaError_t launch_conv_up_dgrad(const Conv3dArgs &g, const void *dy, const void *w_up_t, void *dxa, cudaStream_t st) {
    // K split into 16-channel parts when the collapsed weights of all dy channels do not fit
    const int cs = g.c_out;
    cudaError_t e = cudaErrorNotSupported;
    for (int splits = 1; splits <= cs / 16 && e == cudaErrorNotSupported; splits *= 2) {
        if (cs % splits || (cs / splits) % 16) break;
        e = launch_dwtma(3, g, (const __nv_bfloat16 *)dy, (const __nv_bfloat16 *)w_up_t, nullptr,
                         (__nv_bfloat16 *)dxa, nullptr, cs, g.c_in, 0, st, cs, nullptr, splits);
    }
    return e;
}

cudaError_t launch_collapse_up_t(const void *w, void *w_up_t, int co, int ci, cudaStream_t st) {
    const long long n = (long long)co * 64 * ci;
    conv3_collapse_up_t_kernel<<<grid_for(n), 256, 0, st>>>((const __nv_bfloat16 *)w, (__nv_bfloat16 *)w_up_t, co,
                                                            ci);
    return cudaGetLastError();
}

cudaError_t launch_collapse_up(const void *w, void *w_up, int co, int ci, cudaStream_t st) {
    const long long n = (long long)co * 64 * ci;
    conv3_collapse_up_kernel<<<grid_for(n), 256, 0, st>>>((const __nv_bfloat16 *)w, (__nv_bfloat16 *)w_up, co, ci);
    return cudaGetLastError();
}

cudaError_t launch_conv_halo(const Conv3dArgs &g, const void *src, const void *wt, const float *bias,
                             void *out_bf16, float *out_f32, int Cs, int Nn, int relu, cudaStream_t st,
                             int ca, int up_a, const void *src_b) {
    if (ca <= 0) ca = Cs;
    if (FDC_CONV_DWTMA && FDC_CONV_DWALK && !up_a && Cs <= FDC_CONV_DWALK_MAXC && Cs % 16 == 0 && Nn % 16 == 0) {
        const cudaError_t e = launch_dwtma(0, g, (const __nv_bfloat16 *)src, (const __nv_bfloat16 *)wt, bias,
                                           (__nv_bfloat16 *)out_bf16, out_f32, Cs, Nn, relu, st, ca,
                                           (const __nv_bfloat16 *)src_b);
        if (e != cudaErrorNotSupported) return e;
    }
    // wider inputs (the 32^3 and 16^3 levels' 128 channels): the K dimension split into
    // 64-channel parts on the same kernel, FP32 partial sums combined in order (with a plain
    // ReLU mask for a data gradient)
    if (FDC_CONV_DWTMA && FDC_DWT_KSPLIT && !up_a && g.mask_ca == 0 && !g.out_b && Cs > FDC_CONV_DWALK_MAXC &&
        Cs % FDC_DWT_KSPLIT_CH == 0 && Cs <= 8 * 64 && Nn % 16 == 0) {
        const cudaError_t e = launch_dwtma(0, g, (const __nv_bfloat16 *)src, (const __nv_bfloat16 *)wt, bias,
                                           (__nv_bfloat16 *)out_bf16, out_f32, Cs, Nn, relu, st, ca,
                                           (const __nv_bfloat16 *)src_b, Cs / FDC_DWT_KSPLIT_CH);
        if (e != cudaErrorNotSupported) return e;
    }
    auto s = (const __nv_bfloat16 *)src;
    auto w = (const __nv_bfloat16 *)wt;
    auto ob = (__nv_bfloat16 *)out_bf16;
    auto sb = (const __nv_bfloat16 *)src_b;
    // input channels <= 32 (the 128^3 and 64^3 levels of the network): the
    // d-walking kernel, CTAs spread over the flattened (tile, d) planes
    if (FDC_CONV_DWALK && Cs <= FDC_CONV_DWALK_MAXC && Nn % 16 == 0 &&
        dwalk_fits(Cs / 16, Nn % 32 == 0 ? 32 : 16)) {
        int dev = 0, sms = 0, smem_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (e != cudaSuccess) return e;
        const int S = Cs / 16;
        const int NT = Nn % 32 == 0 ? 32 : 16;
        const int wbytes = S * 9 * 2 * (3 * NT) * 16;
        const int plane = S * kDwPlaneSliceBytes;
        // CTAs per SM are bounded by TMEM (two accumulators of 64 or 128 of the
        // 512 columns): 4 with 16-channel tiles, 2 with 32.  The plane ring
        // takes what shared memory leaves at that residency: 5 to 10 slots
        // (prefetch 1 to 6 planes ahead).
        const int per_sm_tmem = NT == 32 ? 2 : 4;
        const int budget = smem_sm / per_sm_tmem - 2048;
        const int R = std::max(5, std::min(10, (budget - wbytes) / plane));
        const int pf = R - 4;
        const int smem = wbytes + R * plane;
        cudaFuncAttributes fa;
        int per_sm = 0;
        const int thr = (NT == 16 && S == 1) ? 128 : 256;
        if (NT == 32) {
            static OccCache cache;
            e = prepare_kernel_smem(cache, conv3_dwalk_kernel<32, 256>, smem);
            if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, conv3_dwalk_kernel<32, 256>);
        } else if (thr == 128) {
            static OccCache cache;
            e = prepare_kernel_smem(cache, conv3_dwalk_kernel<16, 128>, smem);
            if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, conv3_dwalk_kernel<16, 128>);
        } else {
            static OccCache cache;
            e = prepare_kernel_smem(cache, conv3_dwalk_kernel<16, 256>, smem);
            if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, conv3_dwalk_kernel<16, 256>);
        }
        if (e != cudaSuccess) return e;
        const int by_smem = smem_sm / (smem + (int)fa.sharedSizeBytes + 1024);
        const int by_regs = 65536 / (thr * std::max(fa.numRegs, 1));
        per_sm = std::max(1, std::min(per_sm_tmem, std::min(by_smem, by_regs)));
        const int ntiles = (Nn + NT - 1) / NT;
        const long long planes = (long long)g.batch * ((g.in_h + 7) / 8) * ((g.in_w + 13) / 14) * g.in_d;
        long long gx = std::max(1ll, (long long)sms * per_sm / ntiles);
        if (gx > planes) gx = planes;
        const dim3 grid((unsigned)gx, (unsigned)ntiles);
        if (NT == 32)
            conv3_dwalk_kernel<32, 256><<<grid, 256, smem, st>>>(g, s, w, bias, ob, out_f32, Cs, Nn, relu, ca, up_a, sb, pf);
        else if (thr == 128)
            conv3_dwalk_kernel<16, 128><<<grid, 128, smem, st>>>(g, s, w, bias, ob, out_f32, Cs, Nn, relu, ca, up_a, sb, pf);
        else
            conv3_dwalk_kernel<16, 256><<<grid, 256, smem, st>>>(g, s, w, bias, ob, out_f32, Cs, Nn, relu, ca, up_a, sb, pf);
        return cudaGetLastError();
    }
    // 64-channel tiles (27 MMAs of N = 64) when they give at least one CTA per SM
    // (measured: 32^3 x 64 channels 46 vs 55 us; with 128 input channels at 32^3
    // the kw-stacked 32-channel tiles made U-Net inference 1.24 vs 1.20 ms);
    // otherwise the kw-stacked kernel spreads small grids wider (16^3 x 128: 43 vs 64 us)
    const long long tiles64 = (long long)g.batch * g.in_d * ((g.in_h + 15) / 16) * ((g.in_w + 7) / 8);
    if (FDC_CONV_TC64 && Nn % 64 == 0 && tiles64 * (Nn / 64) >= 152) {
        static OccCache cache;
        const int smem = kTcHaloBytes + 27 * 2 * 64 * 16;
        const cudaError_t e = prepare_kernel_smem(cache, conv3_tc_kernel<64>, smem);
        if (e != cudaSuccess) return e;
        const long long tiles = (long long)g.batch * g.in_d * ((g.in_h + 15) / 16) * ((g.in_w + 7) / 8);
        conv3_tc_kernel<64><<<dim3((unsigned)tiles, (unsigned)(Nn / 64)), 128, smem, st>>>(
            g, s, w, bias, ob, out_f32, Cs, Nn, relu, ca, up_a, sb);
        return cudaGetLastError();
    }
    const long long tiles = (long long)g.batch * g.in_d * ((g.in_h + 7) / 8) * ((g.in_w + 13) / 14);
    // blocks per CTA: enough CTAs for a few waves, weights staged once per CTA
    const int tpc = tiles >= 8 * 152 * 4 ? 4 : (tiles >= 4 * 152 * 2 ? 2 : 1);
    const unsigned grid_x = (unsigned)((tiles + tpc - 1) / tpc);
    if (Nn % 32 == 0 && FDC_KWS_NT != 16) {
        constexpr int kW = 9 * 2 * 96 * 16;
        const int resw = (Cs / 16) * kW <= 56 * 1024;
        const int smem = kKwHaloBytes + (resw ? Cs / 16 : 1) * kW;
        static OccCache cache;
        const cudaError_t e = prepare_kernel_smem(cache, conv3_kws_kernel<32>, smem);
        if (e != cudaSuccess) return e;
        conv3_kws_kernel<32><<<dim3(grid_x, (unsigned)(Nn / 32)), 128, smem, st>>>(
            g, s, w, bias, ob, out_f32, Cs, Nn, relu, ca, up_a, sb, tpc, resw);
    } else {
        constexpr int kW = 9 * 2 * 48 * 16;
        const int resw = (Cs / 16) * kW <= 56 * 1024;
        const int smem = kKwHaloBytes + (resw ? Cs / 16 : 1) * kW;
        static OccCache cache;
        const cudaError_t e = prepare_kernel_smem(cache, conv3_kws_kernel<16>, smem);
        if (e != cudaSuccess) return e;
        conv3_kws_kernel<16><<<dim3(grid_x, (unsigned)(Nn / 16)), 128, smem, st>>>(
            g, s, w, bias, ob, out_f32, Cs, Nn, relu, ca, up_a, sb, tpc, resw);
    }
    return cudaGetLastError();
}

bool conv_dwalk_enabled() { return FDC_CONV_DWALK != 0; }

cudaError_t launch_wait_timeout(long long cycles, cudaStream_t st) {
    wait_timeout_kernel<<<1, 32, 0, st>>>(cycles);
    return cudaGetLastError();
}

int tc_status(bool clear) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_status, sizeof(int)) != cudaSuccess) return (int)FDC_ERR_CUDA;
    if (clear && v) {
        const int z = 0;
        if (cudaMemcpyToSymbol(g_tc_status, &z, sizeof(int)) != cudaSuccess) return (int)FDC_ERR_CUDA;
    }
    return v;
}

cudaError_t launch_flip_transpose(const void *w, void *wf, int co, int k, int ci, cudaStream_t st) {
    const long long n = (long long)co * k * k * k * ci;
    flip_transpose_kernel<<<grid_for(n), 256, 0, st>>>((const __nv_bfloat16 *)w, (__nv_bfloat16 *)wf, co, k, ci);
    return cudaGetLastError();
}

// The down-convolutions on tcgen05 (2^3, stride 2, no padding): returns
// false, launching nothing, for a shape without an instantiation.
template <int MODE, int N, int K>
cudaError_t launch_s2_tc(const Conv3dArgs &g, const void *src, const void *wt, const float *bias, void *out_bf16,
                         float *out_f32, int ntiles_n, cudaStream_t st, const void *residual = nullptr) {
    static OccCache cache;
    constexpr int smem = N * K * 2 + 2 * kS2Vox * K * 2;
    int dev = 0, sms = 0, smem_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = prepare_kernel_smem(cache, conv_s2_tc_kernel<MODE, N, K>, smem);
    if (e != cudaSuccess) return e;
    const int per_sm = std::max(1, std::min(512 / (2 * N), smem_sm / (smem + 2048)));
    const long long tiles = ((long long)g.batch * g.out_d * g.out_h * g.out_w + kS2Vox - 1) / kS2Vox;
    long long gx = std::max(1ll, (long long)sms * per_sm / ntiles_n);
    if (gx > tiles) gx = tiles;
    conv_s2_tc_kernel<MODE, N, K><<<dim3((unsigned)gx, (unsigned)ntiles_n), 128, smem, st>>>(
        g, (const __nv_bfloat16 *)src, (const __nv_bfloat16 *)wt, bias, (__nv_bfloat16 *)out_bf16, out_f32,
        (const __nv_bfloat16 *)residual);
    return cudaGetLastError();
}

// CTAs per SM that the K split of a small mma.sync forward grid aims at
#ifndef FDC_IGEMM_SPLIT_CTAS
#define FDC_IGEMM_SPLIT_CTAS 4
#endif

// widest output-channel tile of the mma.sync forward (its grid is small on
// coarse levels: narrower tiles give more CTAs)
#ifndef FDC_IGEMM_FWD_NT
#define FDC_IGEMM_FWD_NT 32
#endif

bool s2_tc_shape(const Conv3dArgs &g, int mode, const float *out_f32) {
    if (g.ksize != 2 || g.stride != 2 || g.pad != 0) return false;
    if ((long long)g.batch * g.out_d * g.out_h * g.out_w >= (1ll << 31) - kS2Vox) return false;
    if (mode == 0) return (g.c_in == 16 && g.c_out == 32) || (g.c_in == 32 && g.c_out == 64);
    return out_f32 == nullptr && ((g.c_in == 16 && g.c_out == 32) || (g.c_in == 32 && g.c_out == 64) ||
                                  (g.c_in == 64 && g.c_out == 128));
}

cudaError_t launch_conv(const Conv3dArgs &g, int mode, const void *src, const void *wt, const float *bias,
                        void *out_bf16, float *out_f32, cudaStream_t st, const void *residual) {
    const size_t in_bytes = (size_t)g.batch * g.in_d * g.in_h * g.in_w * g.c_in * sizeof(__nv_bfloat16);
    if (s2_tc_shape(g, mode, out_f32)) {
        if (mode == 0) {
            if (g.c_in == 16) return launch_s2_tc<0, 32, 128>(g, src, wt, bias, out_bf16, out_f32, 1, st);
            return launch_s2_tc<0, 64, 256>(g, src, wt, bias, out_bf16, out_f32, 1, st);
        }
        // input voxels of an odd-sized axis's last plane reach no output: their
        // gradient is zero, or the residual
        if ((g.in_d | g.in_h | g.in_w) & 1) {
            const cudaError_t e = residual ? cudaMemcpyAsync(out_bf16, residual, in_bytes, cudaMemcpyDeviceToDevice, st)
                                           : cudaMemsetAsync(out_bf16, 0, in_bytes, st);
            if (e != cudaSuccess) return e;
        }
        if (g.c_in == 16) return launch_s2_tc<1, 128, 32>(g, src, wt, nullptr, out_bf16, nullptr, 1, st, residual);
        if (g.c_in == 32) return launch_s2_tc<1, 256, 64>(g, src, wt, nullptr, out_bf16, nullptr, 1, st, residual);
        return launch_s2_tc<1, 256, 128>(g, src, wt, nullptr, out_bf16, nullptr, 2, st, residual);
    }
    const int Nn = mode == 0 ? g.c_out : g.c_in;
    const long long rows = (long long)g.batch * (mode == 0 ? (long long)g.out_d * g.out_h * g.out_w
                                                          : (long long)g.in_d * g.in_h * g.in_w);
    const int nt_max = mode == 0 ? FDC_IGEMM_FWD_NT : 64;
    const int nt = Nn >= 64 && nt_max >= 64 ? 64 : (Nn >= 32 && nt_max >= 32 ? 32 : 16);
    // data gradient of a tiling convolution: one grid layer per parity class
    const bool par = mode == 1 && g.stride == g.ksize && g.pad == 0;
    const int classes = par ? g.stride * g.stride * g.stride : 1;
    long long rows_c = rows;
    if (par)  // the largest class (parity 0 in every dimension)
        rows_c = (long long)g.batch * ((g.in_d + g.stride - 1) / g.stride) * ((g.in_h + g.stride - 1) / g.stride) *
                 ((g.in_w + g.stride - 1) / g.stride);
    dim3 grid((unsigned)((rows_c + kRows - 1) / kRows), (unsigned)((Nn + nt - 1) / nt), (unsigned)classes);
    auto s = (const __nv_bfloat16 *)src;
    auto w = (const __nv_bfloat16 *)wt;
    auto ob = (__nv_bfloat16 *)out_bf16;
    if (mode == 0) {
        // a grid of fewer than two CTAs per SM (the 32^3 -> 16^3 down-convolution,
        // 64 -> 128 channels: 128 CTAs, each a chain of 32 K steps whose
        // operand loads wait on memory one after the other): K split over
        // grid.z into about four CTAs per SM of at least two K steps each, FP32
        // partials summed in split order by the combine pass, which adds bias
        // and ReLU
        int dev = 0, sms = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        const long long ctas = (long long)grid.x * grid.y;
        const int ksteps = g.ksize * g.ksize * g.ksize * (g.c_in / 16);
        int splits = 1;
        if (ctas < 2ll * sms && Nn % 4 == 0)
            splits = (int)std::min<long long>(ksteps / 2, ((long long)FDC_IGEMM_SPLIT_CTAS * sms + ctas - 1) / ctas);
        if (splits < 1) splits = 1;
        if (splits > 1) {
            const long long n_out = rows * Nn;
            float *part = nullptr;
            e = split_scratch((size_t)n_out * splits, st, &part);
            if (e != cudaSuccess) return e;
            Conv3dArgs gk = g;
            gk.relu = 0;
            grid.z = (unsigned)splits;
            if (nt == 64) conv_igemm_kernel<0, 64><<<grid, 128, 0, st>>>(gk, s, w, nullptr, nullptr, part);
            else if (nt == 32) conv_igemm_kernel<0, 32><<<grid, 128, 0, st>>>(gk, s, w, nullptr, nullptr, part);
            else conv_igemm_kernel<0, 16><<<grid, 128, 0, st>>>(gk, s, w, nullptr, nullptr, part);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            long long blocks = (n_out / 4 + 255) / 256;
            if (blocks > (long long)sms * 16) blocks = (long long)sms * 16;
            split_combine_kernel<<<(int)blocks, 256, 0, st>>>(part, splits, n_out, bias, Nn, g.relu, nullptr,
                                                              ob, out_f32);
            return cudaGetLastError();
        }
        if (nt == 64) conv_igemm_kernel<0, 64><<<grid, 128, 0, st>>>(g, s, w, bias, ob, out_f32);
        else if (nt == 32) conv_igemm_kernel<0, 32><<<grid, 128, 0, st>>>(g, s, w, bias, ob, out_f32);
        else conv_igemm_kernel<0, 16><<<grid, 128, 0, st>>>(g, s, w, bias, ob, out_f32);
    } else {
        if (nt == 64) conv_igemm_kernel<1, 64><<<grid, 128, 0, st>>>(g, s, w, nullptr, ob, out_f32);
        else if (nt == 32) conv_igemm_kernel<1, 32><<<grid, 128, 0, st>>>(g, s, w, nullptr, ob, out_f32);
        else conv_igemm_kernel<1, 16><<<grid, 128, 0, st>>>(g, s, w, nullptr, ob, out_f32);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && residual && mode == 1)
        e = launch_add_bf16(out_bf16, residual, out_bf16, (long long)(in_bytes / sizeof(__nv_bfloat16)), st);
    return e;
}

cudaError_t launch_conv_wgrad(const Conv3dArgs &g, const void *x, const void *dy, float *dw, float *db,
                              cudaStream_t st, int ca, int up_a, const void *xb) {
    if (ca <= 0) ca = g.c_in;
    const long long rows = (long long)g.batch * g.out_d * g.out_h * g.out_w;
    if (g.ksize == 3 && g.stride == 1 && g.pad == 1) {  // tcgen05, voxels as K (c_in, c_out multiples of 16)
        int dev = 0, sms = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        const int vec = ((uintptr_t)dw & 15) == 0 ? 1 : 0;
        auto X = (const __nv_bfloat16 *)x, Y = (const __nv_bfloat16 *)dy, XB = (const __nv_bfloat16 *)xb;
        // 32-channel input slices (M = 128) where the channels allow, else 16 (M = 64);
        // two CTAs per SM (256 TMEM columns, ~94 KB of shared memory each)
        const bool wide = g.c_in % 32 == 0;
        const int cg = wide ? 4 : 2, ht = wide ? 2 : 4, wt = 8;
        const long long chunks = (long long)g.batch * ((g.in_d + kWtDt - 1) / kWtDt) * ((g.in_h + ht - 1) / ht) *
                                 ((g.in_w + wt - 1) / wt);
        if (chunks >= (1ll << 31) || (long long)g.in_d * g.in_h * g.in_w >= (1ll << 31)) return cudaErrorInvalidValue;
        const int ytiles = g.c_out / 16, zslices = g.c_in / (8 * cg);
        long long gx = std::max(1ll, (long long)sms * 2 / (ytiles * zslices));
        if (gx > chunks) gx = chunks;
        const dim3 grid((unsigned)gx, (unsigned)ytiles, (unsigned)zslices);
        if (wide) {
            using P = WgTc<4, 2, 8>;
            static OccCache cache;
            e = prepare_kernel_smem(cache, conv3_wgrad_tc_kernel<4, 2, 8>, P::Smem);
            if (e != cudaSuccess) return e;
            conv3_wgrad_tc_kernel<4, 2, 8><<<grid, kWtThreads, P::Smem, st>>>(g, X, Y, dw, db, ca, up_a, XB, vec);
        } else {
            using P = WgTc<2, 4, 8>;
            static OccCache cache;
            e = prepare_kernel_smem(cache, conv3_wgrad_tc_kernel<2, 4, 8>, P::Smem);
            if (e != cudaSuccess) return e;
            conv3_wgrad_tc_kernel<2, 4, 8><<<grid, kWtThreads, P::Smem, st>>>(g, X, Y, dw, db, ca, up_a, XB, vec);
        }
        return cudaGetLastError();
    }
    const long long vox2 = (long long)g.batch * g.out_d * g.out_h * g.out_w;
    if (g.ksize == 2 && g.stride == 2 && g.pad == 0 && (g.c_out == 32 || g.c_out == 64 || g.c_out == 128) &&
        vox2 < (1ll << 31) - kS2Vox) {  // the down-convolutions: tcgen05, voxels as K
        int dev = 0, sms = 0, smem_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (e != cudaSuccess) return e;
        const int vec = ((uintptr_t)dw & 15) == 0 ? 1 : 0;
        const int smem = 2 * (16 + g.c_out / 8) * kS2Vox * 16;
        const int per_sm = std::max(1, smem_sm / (smem + 2048));
        const long long chunks = (vox2 + kS2Vox - 1) / kS2Vox;
        const int zs = g.c_in / 16;
        long long gx = std::max(1ll, (long long)sms * per_sm / zs);
        if (gx > chunks) gx = chunks;
        const dim3 grid((unsigned)gx, 1, (unsigned)zs);
        auto X = (const __nv_bfloat16 *)x, Y = (const __nv_bfloat16 *)dy;
        static OccCache c32, c64, c128;
        if (g.c_out == 32) {
            e = prepare_kernel_smem(c32, conv_s2_wgrad_tc_kernel<32>, smem);
            if (e == cudaSuccess) conv_s2_wgrad_tc_kernel<32><<<grid, kS2Threads, smem, st>>>(g, X, Y, dw, db, vec);
        } else if (g.c_out == 64) {
            e = prepare_kernel_smem(c64, conv_s2_wgrad_tc_kernel<64>, smem);
            if (e == cudaSuccess) conv_s2_wgrad_tc_kernel<64><<<grid, kS2Threads, smem, st>>>(g, X, Y, dw, db, vec);
        } else {
            e = prepare_kernel_smem(c128, conv_s2_wgrad_tc_kernel<128>, smem);
            if (e == cudaSuccess) conv_s2_wgrad_tc_kernel<128><<<grid, kS2Threads, smem, st>>>(g, X, Y, dw, db, vec);
        }
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    const int taps = g.ksize * g.ksize * g.ksize;
    const int tiles = ((g.c_out + 63) / 64) * ((g.c_in + 63) / 64);
    // enough CTAs to fill the GPU, K chunks of whole 16-voxel steps
    long long chunks = (152ll * 16 + (long long)tiles * taps - 1) / ((long long)tiles * taps);
    if (chunks < 1) chunks = 1;
    long long chunk = (rows + chunks - 1) / chunks;
    chunk = ((chunk + kWgVox - 1) / kWgVox) * kWgVox;
    if (chunk < 256) chunk = 256;
    chunks = (rows + chunk - 1) / chunk;
    dim3 grid((unsigned)tiles, (unsigned)taps, (unsigned)chunks);
    conv_wgrad_kernel<<<grid, 128, 0, st>>>(g, (const __nv_bfloat16 *)x, (const __nv_bfloat16 *)dy, dw, db,
                                            (int)chunk);
    return cudaGetLastError();
}

cudaError_t launch_transpose_weights(const void *w, void *wt, int co, int taps, int ci, cudaStream_t st) {
    const long long n = (long long)co * taps * ci;
    transpose_weights_kernel<<<grid_for(n), 256, 0, st>>>((const __nv_bfloat16 *)w, (__nv_bfloat16 *)wt, co, taps, ci);
    return cudaGetLastError();
}

cudaError_t launch_relu_bwd(const void *y, const void *dy, void *dx, long long n, cudaStream_t st) {
    relu_bwd_kernel<<<grid_for(n), 256, 0, st>>>((const __nv_bfloat16 *)y, (const __nv_bfloat16 *)dy,
                                                 (__nv_bfloat16 *)dx, n);
    return cudaGetLastError();
}

cudaError_t launch_upsample2(const void *x, void *y, int B, int D, int H, int W, int C, int backward,
                             cudaStream_t st) {
    const long long n = (long long)B * D * H * W * C * (backward ? 1 : 8);
    if (backward)
        upsample2_bwd_kernel<<<grid_for(n), 256, 0, st>>>((const __nv_bfloat16 *)x, (__nv_bfloat16 *)y, B, D, H, W, C);
    else
        upsample2_fwd_kernel<<<grid_for(n), 256, 0, st>>>((const __nv_bfloat16 *)x, (__nv_bfloat16 *)y, B, D, H, W, C);
    return cudaGetLastError();
}

cudaError_t launch_concat(const void *a, int Ca, const void *b, int Cb, void *out, long long rows, int inverse,
                          cudaStream_t st) {
    concat_kernel<<<grid_for(rows * (Ca + Cb)), 256, 0, st>>>((const __nv_bfloat16 *)a, Ca, (const __nv_bfloat16 *)b,
                                                             Cb, (__nv_bfloat16 *)out, rows, inverse);
    return cudaGetLastError();
}

cudaError_t launch_mse(const float *pred, int C, const float *target, long long rows, void *grad, float *loss,
                       cudaStream_t st) {
    const int vec = (C % 8 == 0 && ((uintptr_t)grad & 15) == 0) ? 1 : 0;
    mse_kernel<<<grid_for(rows), 256, 0, st>>>(pred, C, target, rows, 1.0f / (float)rows, (__nv_bfloat16 *)grad, loss,
                                               vec);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *p, const float *g, float *m, float *v, void *p_bf16, long long n, float lr, float b1,
                        float b2, float eps, float bc1, float bc2, cudaStream_t st) {
    adam_kernel<<<grid_for(n), 256, 0, st>>>(p, g, m, v, (__nv_bfloat16 *)p_bf16, n, lr, b1, b2, eps, bc1, bc2);
    return cudaGetLastError();
}

cudaError_t launch_add_bf16(const void *a, const void *b, void *out, long long n, cudaStream_t st) {
    add_bf16_kernel<<<grid_for(n), 256, 0, st>>>((const __nv_bfloat16 *)a, (const __nv_bfloat16 *)b,
                                                 (__nv_bfloat16 *)out, n);
    return cudaGetLastError();
}

cudaError_t launch_prepare(const double *dose, const float *density, const double *dose_high, long long n,
                           double inv_scale, float density_scale, void *x, float *dose_in, float *target,
                           cudaStream_t st, const double *scale_dev) {
    prepare_kernel<<<grid_for(n), 256, 0, st>>>(dose, density, dose_high, n, inv_scale, density_scale,
                                                (__nv_bfloat16 *)x, dose_in, target, scale_dev);
    return cudaGetLastError();
}

// The dose scale on the device: max(dose) into *scale (FP64 bits, atomic max
// of non-negative values; 0 when every voxel is 0).
cudaError_t launch_dose_scale(const double *dose, long long n, double *scale, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(scale, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
    long long blocks = (n + 1023) / 1024;
    if (blocks > 152 * 8) blocks = 152 * 8;
    max_kernel<<<(int)blocks, 256, 0, st>>>(dose, n, (unsigned long long *)scale);
    return cudaGetLastError();
}

cudaError_t launch_dihedral(const void *x, const float *t, int D, int H, int W, int code, void *xo, float *to,
                            cudaStream_t st) {
    const long long n = (long long)D * H * W;
    dihedral_kernel<<<grid_for(n), 256, 0, st>>>((const uint4 *)x, t, D, H, W, code, (uint4 *)xo, to);
    return cudaGetLastError();
}

cudaError_t launch_finish(const float *head, const float *dose_in, long long n, double scale, double *dose_out,
                          cudaStream_t st) {
    finish_kernel<<<grid_for(n), 256, 0, st>>>(head, dose_in, n, scale, dose_out);
    return cudaGetLastError();
}

cudaError_t launch_head(const void *x, const void *w, const float *b, long long n, const float *dose_in,
                        double scale, float *y, double *dose_out, cudaStream_t st, const double *scale_dev) {
    head_kernel<<<grid_for(n), 256, 0, st>>>((const __nv_bfloat16 *)x, (const __nv_bfloat16 *)w, b, n, dose_in, scale,
                                             y, dose_out, scale_dev);
    return cudaGetLastError();
}

cudaError_t launch_head_loss(const void *x, const void *w, const float *b, const float *target, long long n,
                             float *loss, void *dx, float *dw, float *db, cudaStream_t st) {
    // a few voxels per thread: the block partials and their atomics stay few
    long long blocks = (n + 256 * 4 - 1) / (256 * 4);
    if (blocks > 152 * 8) blocks = 152 * 8;
    head_loss_kernel<<<(int)blocks, 256, 0, st>>>((const __nv_bfloat16 *)x, (const __nv_bfloat16 *)w, b, target, n,
                                                  1.0f / (float)n, loss, (__nv_bfloat16 *)dx, dw, db);
    return cudaGetLastError();
}

cudaError_t launch_gamma(const double *ref, const double *eval, int D, int H, int W, double sd, double sh, double sw,
                         double dd, double dta, double thr, int radius, float *gamma, unsigned long long *scratch,
                         cudaStream_t st) {
    const long long n = (long long)D * H * W;
    cudaError_t e = cudaMemsetAsync(scratch, 0, 3 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    max_kernel<<<grid_for(n), 256, 0, st>>>(ref, n, scratch);
    gamma_kernel<<<grid_for(n, 128), 128, 0, st>>>(ref, eval, D, H, W, sd, sh, sw, dd, dta, thr, radius, scratch,
                                                  gamma, scratch + 1);
    return cudaGetLastError();
}

cudaError_t launch_f32_to_bf16(const float *x, void *y, long long n, cudaStream_t st) {
    f32_to_bf16_kernel<<<grid_for(n), 256, 0, st>>>(x, (__nv_bfloat16 *)y, n);
    return cudaGetLastError();
}

}  // namespace fdc

// ---------------------------------------------------------------- C ABI
#include <cmath>

#include "fdc_unet.h"

namespace {

bool conv_ok(const fdc_conv3d *g) {
    if (!g || g->batch < 1 || g->c_in < 16 || g->c_out < 16 || g->c_in % 16 || g->c_out % 16) return false;
    if (g->c_in > 2048 || g->c_out > 2048) return false;
    if (g->ksize < 1 || g->ksize > 3 || g->stride < 1 || g->pad < 0) return false;
    const int in[3] = {g->in_d, g->in_h, g->in_w}, out[3] = {g->out_d, g->out_h, g->out_w};
    for (int a = 0; a < 3; ++a) {
        if (in[a] < 1 || out[a] < 1) return false;
        if (out[a] != (in[a] + 2 * g->pad - g->ksize) / g->stride + 1) return false;
    }
    return true;
}

fdc::Conv3dArgs to_args(const fdc_conv3d *g) {
    fdc::Conv3dArgs a;
    a.batch = g->batch;
    a.in_d = g->in_d; a.in_h = g->in_h; a.in_w = g->in_w;
    a.out_d = g->out_d; a.out_h = g->out_h; a.out_w = g->out_w;
    a.c_in = g->c_in; a.c_out = g->c_out;
    a.ksize = g->ksize; a.stride = g->stride; a.pad = g->pad; a.relu = g->relu ? 1 : 0;
    a.mask = nullptr;
    a.mask_b = nullptr;
    a.mask_ca = 0;
    a.mask_up = 0;
    a.out_b = nullptr;
    return a;
}

int rc(cudaError_t e) { return e == cudaSuccess ? FDC_OK : FDC_ERR_CUDA; }

}  // namespace

extern "C" {

bool is_k3s1p1(const fdc_conv3d *g) { return g->ksize == 3 && g->stride == 1 && g->pad == 1; }

int fdc_conv3d_forward(const fdc_conv3d *g, const void *x, const void *w, const float *bias, void *y_bf16,
                       float *y_f32, void *stream) {
    if (!conv_ok(g) || !x || !w || (!y_bf16 && !y_f32)) return FDC_ERR_INVALID;
    if (is_k3s1p1(g))
        return rc(fdc::launch_conv_halo(to_args(g), x, w, bias, y_bf16, y_f32, g->c_in, g->c_out, g->relu ? 1 : 0,
                                        (cudaStream_t)stream, g->c_in, 0, nullptr));
    return rc(fdc::launch_conv(to_args(g), 0, x, w, bias, y_bf16, y_f32, (cudaStream_t)stream));
}

int fdc_conv3d_forward_fused(const fdc_conv3d *g, const void *xa, int32_t ca, int32_t upsample_a, const void *xb,
                             const void *w, const float *bias, void *y_bf16, float *y_f32, void *stream) {
    if (!conv_ok(g) || !is_k3s1p1(g) || !xa || !w || (!y_bf16 && !y_f32)) return FDC_ERR_INVALID;
    if (ca < 16 || ca % 16 || ca > g->c_in || (ca < g->c_in && !xb)) return FDC_ERR_INVALID;
    if (upsample_a && (g->in_d % 2 || g->in_h % 2 || g->in_w % 2)) return FDC_ERR_INVALID;
    return rc(fdc::launch_conv_halo(to_args(g), xa, w, bias, y_bf16, y_f32, g->c_in, g->c_out, g->relu ? 1 : 0,
                                    (cudaStream_t)stream, ca, upsample_a ? 1 : 0, xb));
}

int fdc_conv3d_forward_up(const fdc_conv3d *g, const void *xa, const void *w_up, const float *bias, void *y_bf16,
                          float *y_f32, void *stream) {
    if (!conv_ok(g) || !is_k3s1p1(g) || !xa || !w_up || (!y_bf16 && !y_f32)) return FDC_ERR_INVALID;
    if (g->in_d % 2 || g->in_h % 2 || g->in_w % 2) return FDC_ERR_INVALID;
    const cudaError_t e = fdc::launch_conv_up(to_args(g), xa, w_up, bias, y_bf16, y_f32, g->relu ? 1 : 0,
                                              (cudaStream_t)stream);
    return e == cudaErrorNotSupported ? FDC_ERR_INVALID : rc(e);
}

int fdc_conv3d_backward_data_up(const fdc_conv3d *g, const void *dy, const void *w_up_t, const void *relu_mask,
                                void *dxa, void *stream) {
    if (!conv_ok(g) || !is_k3s1p1(g) || !dy || !w_up_t || !dxa) return FDC_ERR_INVALID;
    if (g->in_d % 2 || g->in_h % 2 || g->in_w % 2) return FDC_ERR_INVALID;
    fdc::Conv3dArgs a = to_args(g);
    a.relu = 0;
    a.mask = relu_mask;
    const cudaError_t e = fdc::launch_conv_up_dgrad(a, dy, w_up_t, dxa, (cudaStream_t)stream);
    return e == cudaErrorNotSupported ? FDC_ERR_INVALID : rc(e);
}

int fdc_conv3d_collapse_up_weights_t(const fdc_conv3d *g, const void *w, void *w_up_t, void *stream) {
    if (!conv_ok(g) || !is_k3s1p1(g) || !w || !w_up_t) return FDC_ERR_INVALID;
    return rc(fdc::launch_collapse_up_t(w, w_up_t, g->c_out, g->c_in, (cudaStream_t)stream));
}

int fdc_conv3d_collapse_up_weights(const fdc_conv3d *g, const void *w, void *w_up, void *stream) {
    if (!conv_ok(g) || !is_k3s1p1(g) || !w || !w_up) return FDC_ERR_INVALID;
    return rc(fdc::launch_collapse_up(w, w_up, g->c_out, g->c_in, (cudaStream_t)stream));
}

int fdc_conv3d_backward_data(const fdc_conv3d *g, const void *dy, const void *w_t, const void *relu_mask, void *dx,
                             void *stream) {
    if (!conv_ok(g) || !dy || !w_t || !dx) return FDC_ERR_INVALID;
    fdc::Conv3dArgs a = to_args(g);
    a.relu = 0;
    a.mask = relu_mask;
    if (is_k3s1p1(g))  // forward convolution of dy with the reflected, transposed weights
        return rc(fdc::launch_conv_halo(a, dy, w_t, nullptr, dx, nullptr, g->c_out, g->c_in, 0,
                                        (cudaStream_t)stream, g->c_out, 0, nullptr));
    return rc(fdc::launch_conv(a, 1, dy, w_t, nullptr, dx, nullptr, (cudaStream_t)stream));
}

int fdc_conv3d_backward_data_add(const fdc_conv3d *g, const void *dy, const void *w_t, const void *relu_mask,
                                 const void *residual, void *dx, void *stream) {
    if (!conv_ok(g) || !dy || !w_t || !dx || !residual || residual == dx) return FDC_ERR_INVALID;
    fdc::Conv3dArgs a = to_args(g);
    a.relu = 0;
    a.mask = relu_mask;
    if (is_k3s1p1(g)) {
        cudaError_t e = fdc::launch_conv_halo(a, dy, w_t, nullptr, dx, nullptr, g->c_out, g->c_in, 0,
                                              (cudaStream_t)stream, g->c_out, 0, nullptr);
        if (e == cudaSuccess)
            e = fdc::launch_add_bf16(dx, residual, dx,
                                     (long long)g->batch * g->in_d * g->in_h * g->in_w * g->c_in, (cudaStream_t)stream);
        return rc(e);
    }
    return rc(fdc::launch_conv(a, 1, dy, w_t, nullptr, dx, nullptr, (cudaStream_t)stream, residual));
}

int fdc_conv3d_backward_weights(const fdc_conv3d *g, const void *x, const void *dy, float *dw, float *db,
                                void *stream) {
    if (!conv_ok(g) || !x || !dy || !dw) return FDC_ERR_INVALID;
    return rc(fdc::launch_conv_wgrad(to_args(g), x, dy, dw, db, (cudaStream_t)stream, g->c_in, 0, nullptr));
}

int fdc_conv3d_backward_weights_fused(const fdc_conv3d *g, const void *xa, int32_t ca, int32_t upsample_a,
                                      const void *xb, const void *dy, float *dw, float *db, void *stream) {
    if (!conv_ok(g) || !is_k3s1p1(g) || !xa || !dy || !dw) return FDC_ERR_INVALID;
    if (ca < 16 || ca % 16 || ca > g->c_in || (ca < g->c_in && !xb)) return FDC_ERR_INVALID;
    if (upsample_a && (g->in_d % 2 || g->in_h % 2 || g->in_w % 2)) return FDC_ERR_INVALID;
    return rc(fdc::launch_conv_wgrad(to_args(g), xa, dy, dw, db, (cudaStream_t)stream, ca, upsample_a ? 1 : 0, xb));
}

int fdc_conv3d_backward_data_fused(const fdc_conv3d *g, const void *dy, const void *w_t, const void *xa, int32_t ca,
                                   int32_t upsample_a, const void *xb, void *dxa, void *dxb, void *stream) {
    if (!conv_ok(g) || !is_k3s1p1(g) || !dy || !w_t || !xa || !dxa) return FDC_ERR_INVALID;
    if (g->c_out > 32 || !fdc::conv_dwalk_enabled()) return FDC_ERR_INVALID;  // the d-walking kernels only
    if (ca < 16 || ca % 16 || ca > g->c_in || (ca < g->c_in && (!xb || !dxb))) return FDC_ERR_INVALID;
    if (upsample_a && (g->in_d % 2 || g->in_h % 2 || g->in_w % 2)) return FDC_ERR_INVALID;
    fdc::Conv3dArgs a = to_args(g);
    a.relu = 0;
    a.mask = xa;
    a.mask_b = ca < g->c_in ? xb : nullptr;
    a.mask_ca = ca;
    a.mask_up = upsample_a ? 1 : 0;
    a.out_b = ca < g->c_in ? dxb : nullptr;
    return rc(fdc::launch_conv_halo(a, dy, w_t, nullptr, dxa, nullptr, g->c_out, g->c_in, 0, (cudaStream_t)stream,
                                    g->c_out, 0, nullptr));
}

int fdc_conv3d_transpose_weights(const fdc_conv3d *g, const void *w, void *w_t, void *stream) {
    if (!conv_ok(g) || !w || !w_t) return FDC_ERR_INVALID;
    if (is_k3s1p1(g))
        return rc(fdc::launch_flip_transpose(w, w_t, g->c_out, 3, g->c_in, (cudaStream_t)stream));
    return rc(fdc::launch_transpose_weights(w, w_t, g->c_out, g->ksize * g->ksize * g->ksize, g->c_in,
                                            (cudaStream_t)stream));
}

int fdc_conv3d_transpose_weights_batch(int32_t n, const fdc_conv3d *g, const void *const *w, void *const *w_t,
                                       void *stream) {
    if (n < 0 || (n > 0 && (!g || !w || !w_t))) return FDC_ERR_INVALID;
    for (int i = 0; i < n; ++i)
        if (!conv_ok(&g[i]) || !w[i] || !w_t[i]) return FDC_ERR_INVALID;
    for (int i0 = 0; i0 < n; i0 += fdc::kTrBatch) {
        fdc::TransposeBatch b;
        b.n = std::min(n - i0, fdc::kTrBatch);
        b.start[0] = 0;
        for (int e = 0; e < b.n; ++e) {
            const fdc_conv3d &ge = g[i0 + e];
            b.w[e] = (const __nv_bfloat16 *)w[i0 + e];
            b.wt[e] = (__nv_bfloat16 *)w_t[i0 + e];
            b.co[e] = ge.c_out;
            b.taps[e] = ge.ksize * ge.ksize * ge.ksize;
            b.ci[e] = ge.c_in;
            b.flip[e] = is_k3s1p1(&ge) ? 1 : 0;
            b.start[e + 1] = b.start[e] + (long long)ge.c_out * b.taps[e] * ge.c_in;
        }
        const long long blocks = std::min(4096ll, std::max(1ll, (b.start[b.n] + 255) / 256));
        fdc::transpose_batch_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(b);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return rc(e);
    }
    return FDC_OK;
}

int fdc_relu_backward(const void *y, const void *dy, void *dx, int64_t n, void *stream) {
    if (!y || !dy || !dx || n < 0) return FDC_ERR_INVALID;
    if (!n) return FDC_OK;
    return rc(fdc::launch_relu_bwd(y, dy, dx, n, (cudaStream_t)stream));
}

int fdc_upsample2(const void *x, void *y, int32_t b, int32_t d, int32_t h, int32_t w, int32_t c, int32_t backward,
                  void *stream) {
    if (!x || !y || b < 1 || d < 1 || h < 1 || w < 1 || c < 1) return FDC_ERR_INVALID;
    return rc(fdc::launch_upsample2(x, y, b, d, h, w, c, backward, (cudaStream_t)stream));
}

int fdc_concat_channels(void *a, int32_t ca, void *b, int32_t cb, void *out, int64_t rows, int32_t split,
                        void *stream) {
    if (!a || !b || !out || ca < 1 || cb < 1 || rows < 0) return FDC_ERR_INVALID;
    if (!rows) return FDC_OK;
    return rc(fdc::launch_concat(a, ca, b, cb, out, rows, split, (cudaStream_t)stream));
}

int fdc_mse(const float *pred, int32_t c, const float *target, int64_t rows, void *grad, float *loss, void *stream) {
    if (!pred || !target || !loss || c < 1 || rows < 1) return FDC_ERR_INVALID;
    return rc(fdc::launch_mse(pred, c, target, rows, grad, loss, (cudaStream_t)stream));
}

int fdc_adam(float *p, const float *g, float *m, float *v, void *p_bf16, int64_t n, float lr, float beta1,
             float beta2, float eps, int32_t step, void *stream) {
    if (!p || !g || !m || !v || n < 0 || step < 1 || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) ||
        !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
        return FDC_ERR_INVALID;
    if (!n) return FDC_OK;
    const float bc1 = 1.0f - powf(beta1, (float)step), bc2 = 1.0f - powf(beta2, (float)step);
    return rc(fdc::launch_adam(p, g, m, v, p_bf16, n, lr, beta1, beta2, eps, bc1, bc2, (cudaStream_t)stream));
}

int fdc_add_bf16(const void *a, const void *b, void *out, int64_t n, void *stream) {
    if (!a || !b || !out || n < 0) return FDC_ERR_INVALID;
    if (!n) return FDC_OK;
    return rc(fdc::launch_add_bf16(a, b, out, n, (cudaStream_t)stream));
}

int fdc_unet_prepare(const double *dose, const float *density, const double *dose_high, int64_t n,
                     double dose_scale, float density_scale, void *x, float *dose_in, float *target,
                     void *stream) {
    if (!dose || !density || !x || !dose_in || n < 1 || !(dose_scale > 0) || (target && !dose_high) ||
        ((uintptr_t)x & 15))
        return FDC_ERR_INVALID;
    return rc(fdc::launch_prepare(dose, density, dose_high, n, 1.0 / dose_scale, density_scale, x, dose_in,
                                  target, (cudaStream_t)stream, nullptr));
}

int fdc_unet_dose_scale(const double *dose, int64_t n, double *scale, void *stream) {
    if (!dose || !scale || n < 1) return FDC_ERR_INVALID;
    return rc(fdc::launch_dose_scale(dose, n, scale, (cudaStream_t)stream));
}

int fdc_unet_prepare_dev(const double *dose, const float *density, int64_t n, const double *scale,
                         float density_scale, void *x, float *dose_in, void *stream) {
    if (!dose || !density || !scale || !x || !dose_in || n < 1 || ((uintptr_t)x & 15)) return FDC_ERR_INVALID;
    return rc(fdc::launch_prepare(dose, density, nullptr, n, 1.0, density_scale, x, dose_in, nullptr,
                                  (cudaStream_t)stream, scale));
}

int fdc_unet_dihedral(const void *x, const float *target, int32_t d, int32_t h, int32_t w, int32_t code,
                      void *x_out, float *target_out, void *stream) {
    if (!x || !x_out || x == (const void *)x_out || d < 1 || h < 1 || w < 1 || code < 0 || code > 7 ||
        ((code & 4) && h != w) || (target && (!target_out || target == target_out)))
        return FDC_ERR_INVALID;
    return rc(fdc::launch_dihedral(x, target, d, h, w, code, x_out, target_out, (cudaStream_t)stream));
}

int fdc_unet_status(int32_t clear) { return fdc::tc_status(clear != 0); }

int fdc_debug_wait_timeout(int64_t cycles, void *stream) {
    if (cycles < 1 || cycles > 4000000000ll) return FDC_ERR_INVALID;
    return rc(fdc::launch_wait_timeout(cycles, (cudaStream_t)stream));
}

int fdc_unet_finish(const float *head, const float *dose_in, int64_t n, double dose_scale, double *dose_out,
                    void *stream) {
    if (!head || !dose_in || !dose_out || n < 1 || !(dose_scale > 0)) return FDC_ERR_INVALID;
    return rc(fdc::launch_finish(head, dose_in, n, dose_scale, dose_out, (cudaStream_t)stream));
}

int fdc_unet_head(const void *x, int32_t c, const void *w, const float *b, int64_t n, const float *dose_in,
                  double dose_scale, float *y, double *dose_out, void *stream) {
    if (!x || !w || !b || c != 16 || n < 1 || (!y && !dose_out) || (dose_out && (!dose_in || !(dose_scale > 0))) ||
        ((uintptr_t)x & 15))
        return FDC_ERR_INVALID;
    return rc(fdc::launch_head(x, w, b, n, dose_in, dose_scale, y, dose_out, (cudaStream_t)stream, nullptr));
}

int fdc_unet_head_dev(const void *x, int32_t c, const void *w, const float *b, int64_t n, const float *dose_in,
                      const double *scale, double *dose_out, void *stream) {
    if (!x || !w || !b || c != 16 || n < 1 || !dose_in || !scale || !dose_out || ((uintptr_t)x & 15))
        return FDC_ERR_INVALID;
    return rc(fdc::launch_head(x, w, b, n, dose_in, 1.0, nullptr, dose_out, (cudaStream_t)stream, scale));
}

int fdc_unet_head_loss(const void *x, int32_t c, const void *w, const float *b, const float *target, int64_t n,
                       float *loss, void *dx, float *dw, float *db, void *stream) {
    if (!x || !w || !b || !target || !loss || c != 16 || n < 1 || (!dw != !db) || ((uintptr_t)x & 15) ||
        ((uintptr_t)dx & 15) || (dx && dx == x))
        return FDC_ERR_INVALID;
    return rc(fdc::launch_head_loss(x, w, b, target, n, loss, dx, dw, db, (cudaStream_t)stream));
}

int fdc_gamma(const double *ref, const double *eval, int32_t d, int32_t h, int32_t w, double sd, double sh, double sw,
              double dose_frac, double dta, double threshold, float *gamma, uint64_t *scratch, double *pass_rate,
              void *stream) {
    if (!ref || !eval || !scratch || d < 1 || h < 1 || w < 1 || !(sd > 0 && sh > 0 && sw > 0) ||
        !(dose_frac > 0) || !(dta > 0) || !(threshold >= 0))
        return FDC_ERR_INVALID;
    const double smin = std::fmin(sd, std::fmin(sh, sw));
    int radius = (int)std::ceil(1.5 * dta / smin);
    if (radius > 8) radius = 8;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = fdc::launch_gamma(ref, eval, d, h, w, sd, sh, sw, dose_frac, dta, threshold, radius, gamma,
                                      (unsigned long long *)scratch, st);
    if (e != cudaSuccess) return FDC_ERR_CUDA;
    if (pass_rate) {
        unsigned long long c[3];
        if (cudaMemcpyAsync(c, scratch, sizeof c, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return FDC_ERR_CUDA;
        *pass_rate = c[1] ? (double)c[2] / (double)c[1] : 0.0;
    }
    return FDC_OK;
}

int fdc_f32_to_bf16(const float *x, void *y, int64_t n, void *stream) {
    if (!x || !y || n < 0) return FDC_ERR_INVALID;
    if (!n) return FDC_OK;
    return rc(fdc::launch_f32_to_bf16(x, y, n, (cudaStream_t)stream));
}

}  // extern "C"
