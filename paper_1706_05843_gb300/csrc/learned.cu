// learned.cu -- kernels of the learned preconditioner: 3^4 convolutions as
// implicit GEMMs on the BF16 tensor cores (FP32 accumulate), their two
// backward passes, activation packing and Adam.
//
// Forward and backward-data (the same product with the mirrored, transposed
// weights): k_conv_tc, on the 5th-generation tensor cores (tcgen05.mma, the
// accumulator in tensor memory), described at the kernel.
// Backward-weights: a CTA owns one tap and a chunk of sites; the product
// dW[tap] = dY^T in_shift (32 x 32, K = sites) is accumulated per warp with
// mma.sync and reduced into the FP32 gradient with atomics.
#include "learned.h"

namespace eofa {

namespace {

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(sdst)), "l"(gsrc));
}
// L1-allocating copy: the neighbour rows of consecutive taps overlap
// almost entirely within a CTA's 128 rows, so they are served from L1
__device__ __forceinline__ void cp_async16_ca(void* sdst, const void* gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(sdst)), "l"(gsrc));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldsm_x4_t(unsigned* r, const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma16816(float* d, const unsigned* a, unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// element offset of 16-byte chunk c of row r in a [rows][32] BF16 tile
__device__ __forceinline__ int swz(int r, int c) { return r * 32 + ((c ^ ((r >> 1) & 3)) << 3); }

struct Coord {
    int x, y, z, t;
};
__device__ __forceinline__ Coord coord_of(const ConvGeom& g, int site) {
    Coord c;
    c.x = site % g.X;
    int r = site / g.X;
    c.y = r % g.Y;
    r /= g.Y;
    c.z = r % g.Z;
    c.t = r / g.Z;
    return c;
}
__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
__device__ __forceinline__ int shifted_site(const ConvGeom& g, const Coord& c, int tap) {
    const int dx = tap % 3 - 1, dy = (tap / 3) % 3 - 1, dz = (tap / 9) % 3 - 1, dt = tap / 27 - 1;
    const int x = wrapi(c.x + dx, g.X), y = wrapi(c.y + dy, g.Y), z = wrapi(c.z + dz, g.Z),
              t = wrapi(c.t + dt, g.T);
    return ((t * g.Z + z) * g.Y + y) * g.X + x;
}

enum Epi { EPI_LEAKY_BF16 = 0, EPI_F32 = 1, EPI_DMASK_BF16 = 2 };

// ---------------------------------------------------------------------------
// The convolution on the 5th-generation tensor cores (tcgen05).
//
// A CTA owns 128 output rows (sites) x 32 output channels: the accumulator
// is a 128-lane x 32-column FP32 block of tensor memory (TMEM), allocated by
// warp 0.  Per tap, the 128 neighbour rows (32 BF16 channels each) and the
// tap's 32 x 32 weight block are copied with cp.async (the rows through L1:
// consecutive taps of a CTA read almost the same rows) into shared memory in
// the tensor cores' canonical K-major layout without swizzle: 8-row x
// 16-byte core matrices, 128 bytes apart along K and 512 bytes apart along
// M (N); two buffers, so the copies of tap t+1 overlap the MMAs of tap t.
// One thread issues the tap's two M128 x N32 x K16 MMAs (kind::f16, BF16 in,
// FP32 accumulate) and commits them to the buffer's mbarrier, which frees
// the buffer for tap t+2.  The epilogue: each warp reads its 32 TMEM lanes
// (its threads' rows) with tcgen05.ld.  Every mbarrier wait is bounded; on
// expiry the CTA records the event in tc_fault, skips its output, frees
// its tensor memory and returns.
// ---------------------------------------------------------------------------
__device__ int g_tc_fault;  // set when a bounded wait of the tcgen05 convolution expired

constexpr int kTcStageA = 128 * 64;  // bytes of one A buffer (128 rows x 32 BF16)
constexpr int kTcStageB = 32 * 64;   // bytes of one B buffer (32 rows x 32 BF16)
// dynamic shared memory of an NST-buffer ring: buffers, NST mbarriers, the TMEM address
constexpr int tc_smem_bytes(int nst) { return nst * (kTcStageA + kTcStageB) + 8 * nst + 16; }
constexpr long kTcSpin = 1L << 22;   // mbarrier polls before a wait counts as expired

// byte offset of 16-byte chunk q (K elements 8q..8q+7) of row r in a
// canonical no-swizzle K-major tile with 4 core matrices along K
__device__ __forceinline__ int tc_off(int r, int q) { return ((r >> 3) * 4 + q) * 128 + (r & 7) * 16; }

// shared-memory matrix descriptor: start, leading (K) and stride (M/N)
// byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ unsigned long long tc_desc(unsigned saddr) {
    const unsigned long long lbo = 128, sbo = 512;
    return (unsigned long long)((saddr >> 4) & 0x3FFF) | (((lbo >> 4) & 0x3FFF) << 16) |
           (((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// instruction descriptor: D FP32, A and B BF16, both K-major, N = 32, M = 128
constexpr unsigned kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mbar_init(unsigned a, unsigned n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(n) : "memory");
}
// true when the phase of the given parity has completed; gives up after kTcSpin polls
__device__ __forceinline__ bool mbar_wait(unsigned a, unsigned parity) {
    for (long i = 0; i < kTcSpin; ++i) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <int EPI, int NST>
__global__ void __launch_bounds__(128) k_conv_tc(const bf16* __restrict__ in, const bf16* __restrict__ W,
                                                 void* __restrict__ out, const bf16* __restrict__ mask, ConvGeom g) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char* sA = tc_smem;                         // [NST][kTcStageA]
    unsigned char* sB = tc_smem + NST * kTcStageA;       // [NST][kTcStageB]
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(sB + NST * kTcStageB);  // [NST]
    unsigned* tmem_slot = reinterpret_cast<unsigned*>(bar + NST);
    __shared__ int s_fault;
    const int tid = threadIdx.x, warp = tid >> 5;
    const long rows = (long)g.V * g.S;
    const long gi = (long)blockIdx.x * 128 + tid;
    const bool rv = gi < rows;
    const int sl = rv ? (int)(gi / g.V) : 0;
    const int site = rv ? (int)(gi - (long)sl * g.V) : 0;
    const Coord c = coord_of(g, site);

    if (tid == 0) {
        for (int b = 0; b < NST; ++b) mbar_init(smem_u32(bar + b), 1);
        s_fault = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tmem_slot;

    auto load_tap = [&](int tap, int buf) {
        unsigned char* a = sA + buf * kTcStageA;
        if (rv) {
            const int ns = shifted_site(g, c, tap);
            const bf16* src = in + ((long)sl * g.V + ns) * kCP;
#pragma unroll
            for (int q = 0; q < 4; ++q) cp_async16_ca(a + tc_off(tid, q), src + q * 8);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) *reinterpret_cast<uint4*>(a + tc_off(tid, q)) = make_uint4(0u, 0u, 0u, 0u);
        }
        const int wr = tid >> 2, wq = tid & 3;
        cp_async16(sB + buf * kTcStageB + tc_off(wr, wq), W + ((long)tap * 32 + wr) * 32 + wq * 8);
        cp_commit();
    };

    // ring of NST buffers: taps 0 .. NST-2 are in flight before the first
    // MMA; tap t + NST - 1 goes into the buffer of tap t - 1 once the MMAs
    // of tap t - 1 have been committed as complete.  Tap t is the
    // (t / NST)-th commit on bar[t % NST] (phase parity (t / NST) & 1).
    bool ok = true;
    for (int t = 0; t < NST - 1; ++t) load_tap(t, t);
    for (int tap = 0; tap < 81; ++tap) {
        const int buf = tap % NST;
        const int nx = tap + NST - 1;
        if (nx < 81) {
            if (tap >= 1) {
                const int pt = tap - 1;
                if (!mbar_wait(smem_u32(bar + pt % NST), (pt / NST) & 1)) ok = false;
            }
            load_tap(nx, nx % NST);
            cp_wait<NST - 1>();
        } else {
            cp_wait<0>();
        }
        // this thread's copies of tap's buffer are visible to the tensor cores
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned a0 = smem_u32(sA + buf * kTcStageA), b0 = smem_u32(sB + buf * kTcStageB);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const unsigned long long ad = tc_desc(a0 + h * 256), bd = tc_desc(b0 + h * 256);
                const unsigned acc = (tap > 0 || h > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(bar + buf))
                         : "memory");
        }
    }
    // the last commit covers every MMA of the CTA
    if (!mbar_wait(smem_u32(bar + 80 % NST), (80 / NST) & 1)) ok = false;
    if (!ok) s_fault = 1;
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!s_fault) {
        unsigned r[32];
        const unsigned taddr = tmem + ((unsigned)(warp * 32) << 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
              "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
              "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (rv) {
            if constexpr (EPI == EPI_F32) {
                float4* o = reinterpret_cast<float4*>(reinterpret_cast<float*>(out) + gi * kCP);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    o[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                       __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
            } else {
                uint4* o = reinterpret_cast<uint4*>(reinterpret_cast<bf16*>(out) + gi * kCP);
                const uint4* mk = reinterpret_cast<const uint4*>(mask + gi * kCP);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint4 mq = make_uint4(0u, 0u, 0u, 0u);
                    if constexpr (EPI == EPI_DMASK_BF16) mq = mk[q];
                    const unsigned* mw = reinterpret_cast<const unsigned*>(&mq);
                    unsigned w[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        float v0 = __uint_as_float(r[8 * q + 2 * e]), v1 = __uint_as_float(r[8 * q + 2 * e + 1]);
                        if constexpr (EPI == EPI_LEAKY_BF16) {
                            v0 = v0 > 0.f ? v0 : kLeaky * v0;
                            v1 = v1 > 0.f ? v1 : kLeaky * v1;
                        } else {
                            const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162*>(&mw[e]);
                            v0 *= __bfloat162float(m.x) > 0.f ? 1.f : kLeaky;
                            v1 *= __bfloat162float(m.y) > 0.f ? 1.f : kLeaky;
                        }
                        const __nv_bfloat162 b = __floats2bfloat162_rn(v0, v1);
                        w[e] = *reinterpret_cast<const unsigned*>(&b);
                    }
                    o[q] = make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
        }
    } else if (tid == 0) {
        atomicExch(&g_tc_fault, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
}

// dW[tap][co][ci] += sum_rows dy[row][co] * in[shift(row, tap)][ci]
__global__ void __launch_bounds__(128) k_conv_wgrad(const bf16* __restrict__ in, const bf16* __restrict__ dy,
                                                    float* __restrict__ dW, ConvGeom g, int cout, int cin,
                                                    int chunk) {
    __shared__ __align__(128) bf16 sD[2][64 * 32];
    __shared__ __align__(128) bf16 sI[2][64 * 32];
    __shared__ float red[4][32 * 33];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tap = blockIdx.y;
    const long rows = (long)g.V * g.S;
    const long k0 = (long)blockIdx.x * chunk;
    const long k1 = k0 + chunk < rows ? k0 + chunk : rows;
    const int nsub = (int)((k1 - k0 + 63) / 64);

    auto load_sub = [&](int sub, int buf) {
        const int r = tid >> 1, q0 = (tid & 1) * 2;
        const long gi = k0 + (long)sub * 64 + r;
        if (gi < k1) {
            const int sl = (int)(gi / g.V);
            const int site = (int)(gi - (long)sl * g.V);
            const int ns = shifted_site(g, coord_of(g, site), tap);
            const bf16* ds = dy + gi * kCP;
            const bf16* is = in + ((long)sl * g.V + ns) * kCP;
#pragma unroll
            for (int q = q0; q < q0 + 2; ++q) {
                cp_async16(sD[buf] + swz(r, q), ds + q * 8);
                cp_async16(sI[buf] + swz(r, q), is + q * 8);
            }
        } else {
#pragma unroll
            for (int q = q0; q < q0 + 2; ++q) {
                *reinterpret_cast<uint4*>(sD[buf] + swz(r, q)) = make_uint4(0u, 0u, 0u, 0u);
                *reinterpret_cast<uint4*>(sI[buf] + swz(r, q)) = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        cp_commit();
    };

    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;

    if (nsub > 0) load_sub(0, 0);
    for (int sub = 0; sub < nsub; ++sub) {
        if (sub + 1 < nsub) {
            load_sub(sub + 1, (sub + 1) & 1);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
        const bf16* D = sD[sub & 1];
        const bf16* In = sI[sub & 1];
        // warp w takes rows (k) w*16 .. w*16+15: one k16 step
        unsigned af[2][4], bfr[2][4];
        const int i = lane >> 3;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {   // A = dy^T: (co, k) from rows k, columns co
            const int r = warp * 16 + (lane & 7) + (i >> 1) * 8;
            ldsm_x4_t(af[mt], D + swz(r, mt * 2 + (i & 1)));
        }
#pragma unroll
        for (int np = 0; np < 2; ++np) {   // B = in_shift: (k, ci) rows k
            const int r = warp * 16 + (lane & 7) + (i & 1) * 8;
            ldsm_x4_t(bfr[np], In + swz(r, np * 2 + (i >> 1)));
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
                mma16816(acc[mt][nt], af[mt], bfr[nt >> 1][(nt & 1) * 2], bfr[nt >> 1][(nt & 1) * 2 + 1]);
        __syncthreads();
    }
    // reduce the 4 warps' partial 32x32 blocks, then one atomic per element
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int co = mt * 16 + (lane >> 2) + h * 8;
                const int ci = nt * 8 + (lane & 3) * 2;
                red[warp][co * 33 + ci] = acc[mt][nt][h * 2];
                red[warp][co * 33 + ci + 1] = acc[mt][nt][h * 2 + 1];
            }
    __syncthreads();
    for (int e = tid; e < 32 * 32; e += 128) {
        const int co = e >> 5, ci = e & 31;
        if (co >= cout || ci >= cin) continue;
        const float v = red[0][co * 33 + ci] + red[1][co * 33 + ci] + red[2][co * 33 + ci] + red[3][co * 33 + ci];
        atomicAdd(dW + ((long)tap * cout + co) * cin + ci, v);
    }
}

// public FP32 weights -> padded BF16 forward and mirrored/transposed backward operands
__global__ void k_convert(const float* __restrict__ Wm, bf16* __restrict__ Wf, bf16* __restrict__ Wb, int cout,
                          int cin) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 81 * 32 * 32) return;
    const int tap = e / 1024, co = (e / 32) % 32, ci = e % 32;
    const float v = (co < cout && ci < cin) ? Wm[((long)tap * cout + co) * cin + ci] : 0.f;
    Wf[e] = __float2bfloat16(v);
    // Wb[80 - tap][ci][co] = W[tap][co][ci]
    Wb[((long)(80 - tap) * 32 + ci) * 32 + co] = __float2bfloat16(v);
}

__global__ void k_pack(const float* __restrict__ in24, bf16* __restrict__ a32, long rows) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * kCP) return;
    const long r = e / kCP;
    const int c = (int)(e % kCP);
    a32[e] = __float2bfloat16(c < 24 ? in24[r * 24 + c] : 0.f);
}

__global__ void k_unpack(const float* __restrict__ out32, float* __restrict__ out24, long rows) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * 24) return;
    const long r = e / 24;
    out24[e] = out32[r * kCP + e % 24];
}

__global__ void k_pad_f32(const float* __restrict__ in24, float* __restrict__ out32, long rows) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * kCP) return;
    const long r = e / kCP;
    const int c = (int)(e % kCP);
    out32[e] = c < 24 ? in24[r * 24 + c] : 0.f;
}

__global__ void k_f32_to_bf16(const float* __restrict__ a, bf16* __restrict__ b, long n) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) b[e] = __float2bfloat16(a[e]);
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gg = g[e];
    const float mm = b1 * m[e] + (1.f - b1) * gg;
    const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    w[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

inline int blocks_for(long n, int bt) { return (int)((n + bt - 1) / bt); }

constexpr int kTcStages = 2;  // deeper rings measured no faster

template <int EPI>
cudaError_t conv(const bf16* in, const bf16* W, void* out, const bf16* mask, const ConvGeom& g, cudaStream_t st) {
    const long rows = (long)g.V * g.S;
    if (rows == 0) return cudaSuccess;
    static_assert(tc_smem_bytes(kTcStages) <= 48 * 1024, "no opt-in shared memory needed");
    k_conv_tc<EPI, kTcStages><<<blocks_for(rows, 128), 128, tc_smem_bytes(kTcStages), st>>>(in, W, out, mask, g);
    return cudaGetLastError();
}

cudaError_t wgrad(const bf16* in, const bf16* dy, float* dW, const ConvGeom& g, int cout, int cin,
                  cudaStream_t st) {
    const long rows = (long)g.V * g.S;
    const int chunk = 4096;
    dim3 grid(blocks_for(rows, chunk), 81);
    k_conv_wgrad<<<grid, 128, 0, st>>>(in, dy, dW, g, cout, cin, chunk);
    return cudaGetLastError();
}

}  // namespace

cudaError_t net_convert(const NetDev& n, cudaStream_t st) {
    long off = 0;
    for (int l = 0; l < kNetLayers; ++l) {
        k_convert<<<blocks_for(81 * 32 * 32, 256), 256, 0, st>>>(n.Wm + off, n.Wf[l], n.Wb[l], kNetCout[l],
                                                                 kNetCin[l]);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        off += kNetLayerW[l];
    }
    return cudaSuccess;
}

cudaError_t net_forward(const NetDev& n, const ConvGeom& g, const bf16* a0, bf16* a1, bf16* a2, float* out,
                        cudaStream_t st) {
    cudaError_t e;
    if ((e = conv<EPI_LEAKY_BF16>(a0, n.Wf[0], a1, nullptr, g, st)) != cudaSuccess) return e;
    if ((e = conv<EPI_LEAKY_BF16>(a1, n.Wf[1], a2, nullptr, g, st)) != cudaSuccess) return e;
    return conv<EPI_F32>(a2, n.Wf[2], out, nullptr, g, st);
}

cudaError_t net_backward(const NetDev& n, const ConvGeom& g, const bf16* a0, const bf16* a1, const bf16* a2,
                         const float* dout, float* dW, float* din, bf16* dob, bf16* d1, bf16* d2,
                         cudaStream_t st) {
    const long rows = (long)g.V * g.S;
    cudaError_t e;
    k_f32_to_bf16<<<blocks_for(rows * kCP, 256), 256, 0, st>>>(dout, dob, rows * kCP);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    float* dW0 = dW;
    float* dW1 = dW + kNetLayerW[0];
    float* dW2 = dW1 + kNetLayerW[1];
    if ((e = wgrad(a2, dob, dW2, g, kNetCout[2], kNetCin[2], st)) != cudaSuccess) return e;
    if ((e = conv<EPI_DMASK_BF16>(dob, n.Wb[2], d2, a2, g, st)) != cudaSuccess) return e;
    if ((e = wgrad(a1, d2, dW1, g, kNetCout[1], kNetCin[1], st)) != cudaSuccess) return e;
    if ((e = conv<EPI_DMASK_BF16>(d2, n.Wb[1], d1, a1, g, st)) != cudaSuccess) return e;
    if ((e = wgrad(a0, d1, dW0, g, kNetCout[0], kNetCin[0], st)) != cudaSuccess) return e;
    if (din) return conv<EPI_F32>(d1, n.Wb[0], din, nullptr, g, st);
    return cudaSuccess;
}

cudaError_t net_fault(int* fault) {
    // read and clear the flag the convolution sets when a bounded wait expired
    cudaError_t e = cudaMemcpyFromSymbol(fault, g_tc_fault, sizeof(int));
    if (e == cudaSuccess && *fault) {
        const int zero = 0;
        e = cudaMemcpyToSymbol(g_tc_fault, &zero, sizeof(int));
    }
    return e;
}

cudaError_t pack_act(const float* in24, bf16* a32, long rows, cudaStream_t st) {
    k_pack<<<blocks_for(rows * kCP, 256), 256, 0, st>>>(in24, a32, rows);
    return cudaGetLastError();
}

cudaError_t unpack_out(const float* out32, float* out24, long rows, cudaStream_t st) {
    k_unpack<<<blocks_for(rows * 24, 256), 256, 0, st>>>(out32, out24, rows);
    return cudaGetLastError();
}

cudaError_t pad_f32(const float* in24, float* out32, long rows, cudaStream_t st) {
    k_pad_f32<<<blocks_for(rows * kCP, 256), 256, 0, st>>>(in24, out32, rows);
    return cudaGetLastError();
}

cudaError_t adam_step(float* w, const float* g, float* m, float* v, long n, float lr, float b1, float b2,
                      float eps, int t, cudaStream_t st) {
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    k_adam<<<blocks_for(n, 256), 256, 0, st>>>(w, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

}  // namespace eofa
