// pipe_peaks.cu -- issue-rate micro-benchmarks that give the roofline
// denominators of the path kernels, measured on the GPU that runs them:
// FP32 FMA (scalar and the f32x2 packed form), the 32x32->64 wide integer
// multiply (and its low and high 32-bit halves alone) and the three-way xor
// of Philox4x32-10, the special-function unit (ex2, lg2, sin, cos, rsqrt,
// sqrt approximations), FP64 FMA, and the FMA-pipe mix of the packed path
// kernel: 15 wide multiplies per 44 f32x2 FMAs, the FMA-pipe work of one
// lane's two paths over one step; and the same FP32 work as scalar FFMAs
// (15 wide multiplies per 88 FFMAs), which shows whether scalar FFMAs run on
// the FMA pipe's light half while its heavy half is busy with a multiply.
//
// Each thread runs kChains independent dependency chains of one instruction
// kind in an unrolled loop, so that with enough resident warps the pipe, not
// the latency of a chain, bounds the rate.  The special-function chains put
// one FP32 FMA between two calls to keep the argument in range; that FMA goes
// to a pipe with eight times the special-function unit's throughput.  The
// caller times a launch with CUDA events and divides the executed
// thread-instructions of the measured kind (pipe_peak_launch's return) by it.
// Built as its own library (libpipepeaks.so); nothing on the pricing path
// uses it.
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int kChains = 8;       // independent chains per thread
constexpr int kUnroll = 8;       // chain steps per loop iteration

enum Kind {
    K_FFMA = 0, K_FFMA2 = 1, K_IMAD_WIDE = 2, K_LOP3 = 3, K_EX2 = 4, K_LG2 = 5, K_SIN = 6,
    K_COS = 7, K_RSQRT = 8, K_SQRT = 9, K_DFMA = 10, K_IMAD_LO = 11, K_IMAD_HI = 12, K_MIX = 13,
    K_MIX_SCALAR = 14, K_COUNT = 15
};
constexpr int kMixInstsPerUnit = 59;     // 15 wide multiplies + 44 f32x2 FMAs
constexpr int kMixScalarInstsPerUnit = 103;  // 15 wide multiplies + 88 FFMAs

__device__ __forceinline__ float mufu(int kind, float x)
{
    float y;
    switch (kind) {
    case K_EX2:   asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); break;
    case K_LG2:   asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); break;
    case K_SIN:   asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); break;
    case K_COS:   asm volatile("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); break;
    case K_RSQRT: asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); break;
    default:      asm volatile("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); break;
    }
    return y;
}

// Argument maps that keep each special-function chain finite:
// ex2(0.1 - x/2), lg2(2 + x/4), sin/cos(0.25 + 1.5x), rsqrt/sqrt(1 + x/2).
__device__ __forceinline__ void mufu_map(int kind, float &a, float &b)
{
    switch (kind) {
    case K_EX2: a = -0.5f; b = 0.1f; break;
    case K_LG2: a = 0.25f; b = 2.0f; break;
    case K_SIN: case K_COS: a = 1.5f; b = 0.25f; break;
    default: a = 0.5f; b = 1.0f; break;
    }
}

template <int KIND>
__global__ void peak_kernel(uint32_t iters, float fa, float fb, float *sink)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (KIND == K_FFMA) {
        float x[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = 1.0f + 1e-3f * (float)(tid + i);
        for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
                for (int i = 0; i < kChains; ++i) x[i] = __fmaf_rn(x[i], fa, fb);
            }
        }
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += x[i];
        if (s == 1234.5f) sink[0] = s;
    } else if constexpr (KIND == K_FFMA2) {
        float2 x[kChains];
        const float2 a = make_float2(fa, fa), b = make_float2(fb, fb);
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = make_float2(1.0f + 1e-3f * (float)(tid + i), 1.0f);
        for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
                for (int i = 0; i < kChains; ++i) x[i] = __ffma2_rn(x[i], a, b);
            }
        }
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += x[i].x + x[i].y;
        if (s == 1234.5f) sink[0] = s;
    } else if constexpr (KIND == K_IMAD_WIDE) {
        // d = lo(d) * M + d: the 32x32->64 multiply of a Philox round, chained
        unsigned long long d[kChains];
        const uint32_t m = 0xD2511F53u ^ (uint32_t)__float_as_uint(fa);
#pragma unroll
        for (int i = 0; i < kChains; ++i) d[i] = tid * 2654435761ull + (unsigned long long)i;
        for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
                for (int i = 0; i < kChains; ++i)
                    asm volatile("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d[i]) : "r"((uint32_t)d[i]), "r"(m), "l"(d[i]));
            }
        }
        unsigned long long s = 0;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s ^= d[i];
        if (s == 12345ull) sink[0] = (float)s;
    } else if constexpr (KIND == K_LOP3) {
        // three-way xor, as in a Philox round
        uint32_t x[kChains];
        const uint32_t y = 0x9E3779B9u ^ __float_as_uint(fa), z = 0xBB67AE85u ^ __float_as_uint(fb);
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = tid * 747796405u + (uint32_t)i;
        for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
                for (int i = 0; i < kChains; ++i)
                    asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(x[i]) : "r"(x[i]), "r"(y), "r"(z));
            }
        }
        uint32_t s = 0;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += x[i];
        if (s == 12345u) sink[0] = (float)s;
    } else if constexpr (KIND == K_IMAD_LO || KIND == K_IMAD_HI) {
        // x = lo(x m) + c, or x = hi(x m) + c: each half of the wide multiply alone
        uint32_t x[kChains];
        const uint32_t m = 0xCD9E8D57u ^ __float_as_uint(fa), c = 0x9E3779B9u ^ __float_as_uint(fb);
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = tid * 747796405u + (uint32_t)i;
        for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
                for (int i = 0; i < kChains; ++i) {
                    if constexpr (KIND == K_IMAD_LO)
                        asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(x[i]) : "r"(x[i]), "r"(m), "r"(c));
                    else
                        asm volatile("mad.hi.u32 %0, %1, %2, %3;" : "=r"(x[i]) : "r"(x[i]), "r"(m), "r"(c));
                }
            }
        }
        uint32_t s = 0;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += x[i];
        if (s == 12345u) sink[0] = (float)s;
    } else if constexpr (KIND == K_MIX) {
        // per loop iteration kUnroll mix units of 15 wide multiplies and 44
        // f32x2 FMAs on independent chains, each unit in three parts of 5 wide
        // multiplies and 15, 15 and 14 f32x2 FMAs
        unsigned long long d[5];
        float2 x[15];
        const uint32_t m = 0xD2511F53u ^ (uint32_t)__float_as_uint(fa);
        const float2 a = make_float2(fa, fa), b = make_float2(fb, fb);
#pragma unroll
        for (int i = 0; i < 5; ++i) d[i] = tid * 2654435761ull + (unsigned long long)i;
#pragma unroll
        for (int i = 0; i < 15; ++i) x[i] = make_float2(1.0f + 1e-3f * (float)(tid + i), 1.0f);
        for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < 3 * kUnroll; ++u) {
#pragma unroll
                for (int i = 0; i < 15; ++i) {
                    if (i < 14 || u % 3 != 2) x[i] = __ffma2_rn(x[i], a, b);
                    if (i < 5)
                        asm volatile("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d[i]) : "r"((uint32_t)d[i]), "r"(m), "l"(d[i]));
                }
            }
        }
        unsigned long long s = 0;
        float f = 0.0f;
#pragma unroll
        for (int i = 0; i < 5; ++i) s ^= d[i];
#pragma unroll
        for (int i = 0; i < 15; ++i) f += x[i].x + x[i].y;
        if (s == 12345ull || f == 1234.5f) sink[0] = f + (float)s;
    } else if constexpr (KIND == K_MIX_SCALAR) {
        // per loop iteration kUnroll units of 15 wide multiplies and 88 FFMAs
        // on independent chains, each unit in three parts of 5 wide multiplies
        // and 30, 30 and 28 FFMAs
        unsigned long long d[5];
        float x[30];
        const uint32_t m = 0xD2511F53u ^ (uint32_t)__float_as_uint(fa);
#pragma unroll
        for (int i = 0; i < 5; ++i) d[i] = tid * 2654435761ull + (unsigned long long)i;
#pragma unroll
        for (int i = 0; i < 30; ++i) x[i] = 1.0f + 1e-3f * (float)(tid + i);
        for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < 3 * kUnroll; ++u) {
#pragma unroll
                for (int i = 0; i < 30; ++i) {
                    if (i < 28 || u % 3 != 2) x[i] = __fmaf_rn(x[i], fa, fb);
                    if (i < 5)
                        asm volatile("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d[i]) : "r"((uint32_t)d[i]), "r"(m), "l"(d[i]));
                }
            }
        }
        unsigned long long s = 0;
        float f = 0.0f;
#pragma unroll
        for (int i = 0; i < 5; ++i) s ^= d[i];
#pragma unroll
        for (int i = 0; i < 30; ++i) f += x[i];
        if (s == 12345ull || f == 1234.5f) sink[0] = f + (float)s;
    } else if constexpr (KIND == K_DFMA) {
        double x[kChains];
        const double a = (double)fa, b = (double)fb;
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = 1.0 + 1e-3 * (double)(tid + i);
        for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
                for (int i = 0; i < kChains; ++i) x[i] = __fma_rn(x[i], a, b);
            }
        }
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += x[i];
        if (s == 1234.5) sink[0] = (float)s;
    } else {
        float a, b;
        mufu_map(KIND, a, b);
        float x[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = 0.5f + 1e-3f * (float)((tid + i) & 255);
        for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
                for (int i = 0; i < kChains; ++i) x[i] = mufu(KIND, __fmaf_rn(x[i], a, b));
            }
        }
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += x[i];
        if (s == 1234.5f) sink[0] = s;
    }
}

template <int KIND>
cudaError_t launch_kind(uint32_t blocks, uint32_t threads, uint32_t iters, cudaStream_t st, float *sink)
{
    // fa, fb: FMA chains contract towards 1 (x = 0.999 x + 0.001)
    peak_kernel<KIND><<<blocks, threads, 0, st>>>(iters, 0.999f, 0.001f, sink);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

// Number of instruction kinds; kind k's name is pipe_peak_name(k).
int pipe_peak_kinds(void) { return K_COUNT; }

const char *pipe_peak_name(int kind)
{
    static const char *names[K_COUNT] = {"ffma", "ffma2", "imad_wide", "lop3", "mufu_ex2", "mufu_lg2",
                                         "mufu_sin", "mufu_cos", "mufu_rsqrt", "mufu_sqrt", "dfma",
                                         "imad_lo", "imad_hi", "heavy_mix", "scalar_mix"};
    return (kind >= 0 && kind < K_COUNT) ? names[kind] : "";
}

// Enqueue one launch of kind `kind` on `stream` (cudaStream_t or NULL) with
// `blocks` x `threads` threads and `iters` loop iterations; d_sink is a device
// float that the kernel writes only in a case that never happens.  Writes
// the executed thread-instructions of the measured kind to *thread_insts (for
// the mixes, 59 per unit of 15 wide multiplies and 44 f32x2 FMAs and 103 per
// unit of 15 wide multiplies and 88 FFMAs).
// Returns 0, or -1 for bad arguments, -2 for a launch error.
int pipe_peak_launch(int kind, uint32_t blocks, uint32_t threads, uint32_t iters, void *stream,
                     float *d_sink, double *thread_insts)
{
    if (kind < 0 || kind >= K_COUNT || blocks == 0 || threads == 0 || threads > 1024 || !d_sink ||
        !thread_insts)
        return -1;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    switch (kind) {
    case K_FFMA: e = launch_kind<K_FFMA>(blocks, threads, iters, st, d_sink); break;
    case K_FFMA2: e = launch_kind<K_FFMA2>(blocks, threads, iters, st, d_sink); break;
    case K_IMAD_WIDE: e = launch_kind<K_IMAD_WIDE>(blocks, threads, iters, st, d_sink); break;
    case K_LOP3: e = launch_kind<K_LOP3>(blocks, threads, iters, st, d_sink); break;
    case K_EX2: e = launch_kind<K_EX2>(blocks, threads, iters, st, d_sink); break;
    case K_LG2: e = launch_kind<K_LG2>(blocks, threads, iters, st, d_sink); break;
    case K_SIN: e = launch_kind<K_SIN>(blocks, threads, iters, st, d_sink); break;
    case K_COS: e = launch_kind<K_COS>(blocks, threads, iters, st, d_sink); break;
    case K_RSQRT: e = launch_kind<K_RSQRT>(blocks, threads, iters, st, d_sink); break;
    case K_SQRT: e = launch_kind<K_SQRT>(blocks, threads, iters, st, d_sink); break;
    case K_DFMA: e = launch_kind<K_DFMA>(blocks, threads, iters, st, d_sink); break;
    case K_IMAD_LO: e = launch_kind<K_IMAD_LO>(blocks, threads, iters, st, d_sink); break;
    case K_IMAD_HI: e = launch_kind<K_IMAD_HI>(blocks, threads, iters, st, d_sink); break;
    case K_MIX: e = launch_kind<K_MIX>(blocks, threads, iters, st, d_sink); break;
    default: e = launch_kind<K_MIX_SCALAR>(blocks, threads, iters, st, d_sink); break;
    }
    if (e != cudaSuccess) return -2;
    // the mix: kUnroll units per iteration, kMixInstsPerUnit instructions per unit
    const double per_iter = kind == K_MIX ? (double)kUnroll * kMixInstsPerUnit
                          : kind == K_MIX_SCALAR ? (double)kUnroll * kMixScalarInstsPerUnit
                          : (double)kUnroll * kChains;
    *thread_insts = (double)blocks * threads * (double)iters * per_iter;
    return 0;
}

}  // extern "C"
