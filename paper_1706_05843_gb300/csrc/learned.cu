// learned.cu -- kernels of the learned preconditioner: 3^4 convolutions as
// implicit GEMMs on the BF16 tensor cores (FP32 accumulate), their two
// backward passes, activation packing and Adam.
//
// Forward (and backward-data, which is the same product with the mirrored,
// transposed weights): a CTA owns 128 output sites x 32 output channels;
// the K loop runs over the 81 taps x 32 input channels.  Per tap the 128
// neighbour rows (64 bytes of BF16 channels each) and the tap's 32x32
// weight block are brought to shared memory with cp.async, double buffered,
// in an XOR-swizzled layout that ldmatrix reads without bank conflicts; each
// of the 4 warps runs mma.m16n8k16 on 32 sites x 32 channels.
// Backward-weights: a CTA owns one tap and a chunk of sites; the product
// dW[tap] = dY^T in_shift (32 x 32, K = sites) is accumulated per warp and
// reduced into the FP32 gradient with atomics.
#include "learned.h"

namespace eofa {

namespace {

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(sdst)), "l"(gsrc));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldsm_x4(unsigned* r, const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
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

template <int EPI>
__global__ void __launch_bounds__(128) k_conv(const bf16* __restrict__ in, const bf16* __restrict__ W,
                                              void* __restrict__ out, const bf16* __restrict__ mask, ConvGeom g) {
    __shared__ __align__(128) bf16 sA[2][128 * 32];
    __shared__ __align__(128) bf16 sB[2][32 * 32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long rows = (long)g.V * g.S;
    const long g0 = (long)blockIdx.x * 128;
    const long gi = g0 + tid;
    const bool rv = gi < rows;
    const int sl = rv ? (int)(gi / g.V) : 0;
    const int site = rv ? (int)(gi - (long)sl * g.V) : 0;
    const Coord c = coord_of(g, site);

    auto load_tap = [&](int tap, int buf) {
        bf16* arow = sA[buf];
        if (rv) {
            const int ns = shifted_site(g, c, tap);
            const bf16* src = in + ((long)sl * g.V + ns) * kCP;
#pragma unroll
            for (int q = 0; q < 4; ++q) cp_async16(arow + swz(tid, q), src + q * 8);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                *reinterpret_cast<uint4*>(arow + swz(tid, q)) = make_uint4(0u, 0u, 0u, 0u);
        }
        const int wr = tid >> 2, wq = tid & 3;
        cp_async16(sB[buf] + swz(wr, wq), W + ((long)tap * 32 + wr) * 32 + wq * 8);
        cp_commit();
    };

    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;

    load_tap(0, 0);
    for (int tap = 0; tap < 81; ++tap) {
        if (tap + 1 < 81) {
            load_tap(tap + 1, (tap + 1) & 1);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
        const bf16* A = sA[tap & 1];
        const bf16* B = sB[tap & 1];
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            unsigned af[2][4], bfr[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int r = warp * 32 + mt * 16 + (lane & 15);
                ldsm_x4(af[mt], A + swz(r, ks * 2 + (lane >> 4)));
            }
#pragma unroll
            for (int np = 0; np < 2; ++np) {
                const int r = np * 16 + (lane & 7) + ((lane >> 4) << 3);
                ldsm_x4(bfr[np], B + swz(r, ks * 2 + ((lane >> 3) & 1)));
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
                    mma16816(acc[mt][nt], af[mt], bfr[nt >> 1][(nt & 1) * 2], bfr[nt >> 1][(nt & 1) * 2 + 1]);
        }
        __syncthreads();
    }
    // epilogue: accumulator (row lane/4 [+8], cols 2*(lane%4) [+1]) of each tile
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const long go = g0 + warp * 32 + mt * 16 + (lane >> 2) + h * 8;
            if (go >= rows) continue;
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int col = nt * 8 + (lane & 3) * 2;
                float v0 = acc[mt][nt][h * 2], v1 = acc[mt][nt][h * 2 + 1];
                if constexpr (EPI == EPI_F32) {
                    *reinterpret_cast<float2*>(reinterpret_cast<float*>(out) + go * kCP + col) = make_float2(v0, v1);
                } else {
                    if constexpr (EPI == EPI_LEAKY_BF16) {
                        v0 = v0 > 0.f ? v0 : kLeaky * v0;
                        v1 = v1 > 0.f ? v1 : kLeaky * v1;
                    } else {
                        const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162*>(mask + go * kCP + col);
                        v0 *= __bfloat162float(m.x) > 0.f ? 1.f : kLeaky;
                        v1 *= __bfloat162float(m.y) > 0.f ? 1.f : kLeaky;
                    }
                    *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<bf16*>(out) + go * kCP + col) =
                        __floats2bfloat162_rn(v0, v1);
                }
            }
        }
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

template <int EPI>
cudaError_t conv(const bf16* in, const bf16* W, void* out, const bf16* mask, const ConvGeom& g, cudaStream_t st) {
    const long rows = (long)g.V * g.S;
    if (rows == 0) return cudaSuccess;
    k_conv<EPI><<<blocks_for(rows, 128), 128, 0, st>>>(in, W, out, mask, g);
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
