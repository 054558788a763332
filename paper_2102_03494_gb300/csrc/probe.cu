// probe.cu -- microbenchmark of the GPU's 64 x 64 -> 128-bit multiply-accumulate rate, the
// operation the key-switch, plaintext-product and base-conversion kernels are built from.
//
// The forms, registers only, eight independent accumulators per thread:
//   chain: mac128 (he_internal.cuh), the 32-bit multiply-add carry chain of the Montgomery
//          reductions; chain_wide: mac128r, the 64-bit add-with-carry form of the residue
//          products in the tap, inner-product and MAC kernels;
//   cols:  the same product as four 32 x 32 -> 64-bit partial products summed into three
//          64-bit column accumulators (operands below 2^60 split at bit 30), no carry chain.
// Each iteration also advances one operand (so nothing is loop-invariant); every thread
// writes one word so that no work is dead.
#include "he_internal.cuh"

namespace {

constexpr int kAcc = 8;

// WIDE: mac128r (64-bit add-with-carry of four 32 x 32 -> 64-bit products, operands below
// 2^63, the form the tap, inner-product and MAC kernels use); else mac128.
template <bool WIDE>
__global__ void __launch_bounds__(256) k_probe_chain(const uint64_t* __restrict__ in,
                                                     uint64_t* __restrict__ out, int iters) {
    uint64_t x[kAcc], y[kAcc];
    U128 acc[kAcc];
#pragma unroll
    for (int a = 0; a < kAcc; ++a) {
        x[a] = in[a] + threadIdx.x;
        y[a] = in[kAcc + a];
        acc[a] = U128{0, 0};
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int a = 0; a < kAcc; ++a) {
            if (WIDE) mac128r(acc[a], x[a], y[a]);
            else mac128(acc[a], x[a], y[a]);
            x[a] ^= (uint32_t)i;                  // stays below 2^60 (low word only)
        }
    }
    uint64_t r = 0;
#pragma unroll
    for (int a = 0; a < kAcc; ++a) r ^= acc[a].lo ^ acc[a].hi;
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
}

__global__ void __launch_bounds__(256) k_probe_cols(const uint64_t* __restrict__ in,
                                                    uint64_t* __restrict__ out, int iters) {
    uint32_t x0[kAcc], x1[kAcc], y0[kAcc], y1[kAcc];
    uint64_t c0[kAcc], c1[kAcc], c2[kAcc];
    const uint64_t m60 = (1ull << 60) - 1;
#pragma unroll
    for (int a = 0; a < kAcc; ++a) {
        const uint64_t xv = (in[a] + threadIdx.x) & m60, yv = in[kAcc + a] & m60;
        x0[a] = (uint32_t)(xv & 0x3fffffff);
        x1[a] = (uint32_t)(xv >> 30);
        y0[a] = (uint32_t)(yv & 0x3fffffff);
        y1[a] = (uint32_t)(yv >> 30);
        c0[a] = c1[a] = c2[a] = 0;
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int a = 0; a < kAcc; ++a) {
            c0[a] += (uint64_t)x0[a] * y0[a];
            c1[a] += (uint64_t)x0[a] * y1[a];
            c1[a] += (uint64_t)x1[a] * y0[a];
            c2[a] += (uint64_t)x1[a] * y1[a];
            x0[a] = (x0[a] + y0[a]) & 0x3fffffff;
        }
    }
    uint64_t r = 0;
#pragma unroll
    for (int a = 0; a < kAcc; ++a) r ^= c0[a] ^ c1[a] ^ c2[a];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// Karatsuba form: a b = a0 b0 + ((a0 + a1)(b0 + b1) - a0 b0 - a1 b1) 2^30 + a1 b1 2^60, three
// 32 x 32 -> 64-bit products per 64-bit product; the middle column is formed from the three
// sums once, at the end.
__global__ void __launch_bounds__(256) k_probe_kara(const uint64_t* __restrict__ in,
                                                    uint64_t* __restrict__ out, int iters) {
    uint32_t x0[kAcc], x1[kAcc], y0[kAcc], y1[kAcc];
    uint64_t c0[kAcc], cm[kAcc], c2[kAcc];
    const uint64_t m60 = (1ull << 60) - 1;
#pragma unroll
    for (int a = 0; a < kAcc; ++a) {
        const uint64_t xv = (in[a] + threadIdx.x) & m60, yv = in[kAcc + a] & m60;
        x0[a] = (uint32_t)(xv & 0x3fffffff);
        x1[a] = (uint32_t)(xv >> 30);
        y0[a] = (uint32_t)(yv & 0x3fffffff);
        y1[a] = (uint32_t)(yv >> 30);
        c0[a] = cm[a] = c2[a] = 0;
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int a = 0; a < kAcc; ++a) {
            const uint32_t xs = x0[a] + x1[a], ys = y0[a] + y1[a];
            c0[a] += (uint64_t)x0[a] * y0[a];
            cm[a] += (uint64_t)xs * ys;
            c2[a] += (uint64_t)x1[a] * y1[a];
            x0[a] = (x0[a] + y0[a]) & 0x3fffffff;
        }
    }
    uint64_t r = 0;
#pragma unroll
    for (int a = 0; a < kAcc; ++a) r ^= c0[a] ^ (cm[a] - c0[a] - c2[a]) ^ c2[a];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// Single-instruction streams: eight independent accumulators per thread, each step one
// instruction of the kind measured (op 0: mad.lo.u32, 1: mad.hi.u32, 2: mad.wide.u32).
template <int OP>
__global__ void __launch_bounds__(256) k_probe_op(const uint64_t* __restrict__ in,
                                                  uint64_t* __restrict__ out, int iters) {
    uint32_t acc[kAcc], b[kAcc];
    uint64_t w[kAcc];
#pragma unroll
    for (int a = 0; a < kAcc; ++a) {
        acc[a] = (uint32_t)in[a] + threadIdx.x;
        b[a] = (uint32_t)in[kAcc + a] | 1u;
        w[a] = in[a] ^ threadIdx.x;
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int a = 0; a < kAcc; ++a) {
            if (OP == 0) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(acc[a]) : "r"(b[a]), "r"(b[(a + 1) % kAcc]));
            if (OP == 1) asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(acc[a]) : "r"(b[a]), "r"(b[(a + 1) % kAcc]));
            if (OP == 2) asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(w[a]) : "r"(acc[a]), "r"(b[a]));
        }
    }
    uint64_t r = 0;
#pragma unroll
    for (int a = 0; a < kAcc; ++a) r ^= acc[a] ^ w[a];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// Read bandwidth: every thread streams 16-byte loads that bypass L1 (ld.global.cg) over a
// buffer, `reps` times; a buffer that fits in L2 measures L2, a larger one HBM.
__global__ void __launch_bounds__(256) k_probe_read(const uint4* __restrict__ in, size_t n16,
                                                    int reps, uint64_t* __restrict__ out) {
    uint32_t acc = 0;
    for (int r = 0; r < reps; ++r)
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16;
             i += (size_t)gridDim.x * blockDim.x) {
            const uint4 v = __ldcg(in + i);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    if (acc == 0x9e3779b9u) out[0] = acc;           // keeps the loads live
}

}  // namespace

extern "C" int he_probe_int_mac(he_ctx* ctx, double* out) {
    if (!ctx || !out) return HE_EINVAL;
    HE_NOT_RECORDING(ctx, "he_probe_int_mac");
    int sms = 0, dev = 0;
    HE_CHECK_CUDA(ctx, cudaGetDevice(&dev));
    HE_CHECK_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256, iters = 4096;
    int rc = arena_reserve(ctx, 2 * kAcc + (size_t)blocks * threads + 64);
    if (rc) return rc;
    arena_reset(ctx);
    uint64_t* in = arena_take(ctx, 2 * kAcc);
    uint64_t* o = arena_take(ctx, (size_t)blocks * threads);
    uint64_t h[2 * kAcc];
    for (int i = 0; i < 2 * kAcc; ++i) h[i] = (0x0123456789abcdefull * (i + 1)) & ((1ull << 59) - 1);
    HE_CHECK_CUDA(ctx, cudaMemcpyAsync(in, h, sizeof(h), cudaMemcpyHostToDevice, ctx->stream));
    cudaEvent_t e0, e1;
    HE_CHECK_CUDA(ctx, cudaEventCreate(&e0));
    HE_CHECK_CUDA(ctx, cudaEventCreate(&e1));
    const double prods = (double)blocks * threads * iters * kAcc;
    for (int v = 0; v < 2; ++v) {
        for (int rep = 0; rep < 2; ++rep) {                       // warm-up
            ++ctx->launches;
            if (v == 0) k_probe_chain<false><<<blocks, threads, 0, ctx->stream>>>(in, o, iters);
            else k_probe_cols<<<blocks, threads, 0, ctx->stream>>>(in, o, iters);
        }
        cudaEventRecord(e0, ctx->stream);
        for (int rep = 0; rep < 5; ++rep) {
            ++ctx->launches;
            if (v == 0) k_probe_chain<false><<<blocks, threads, 0, ctx->stream>>>(in, o, iters);
            else k_probe_cols<<<blocks, threads, 0, ctx->stream>>>(in, o, iters);
        }
        cudaEventRecord(e1, ctx->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        out[v] = prods * 5 / (ms / 1e3);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return he_launch_check(ctx, "he_probe_int_mac");
}

extern "C" int he_probe_int_ops(he_ctx* ctx, double* out, int n) {
    if (!ctx || !out || n < 1) return HE_EINVAL;
    HE_NOT_RECORDING(ctx, "he_probe_int_ops");
    int sms = 0, dev = 0;
    HE_CHECK_CUDA(ctx, cudaGetDevice(&dev));
    HE_CHECK_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256, iters = 4096;
    int rc = arena_reserve(ctx, 2 * kAcc + (size_t)blocks * threads + 64);
    if (rc) return rc;
    arena_reset(ctx);
    uint64_t* in = arena_take(ctx, 2 * kAcc);
    uint64_t* o = arena_take(ctx, (size_t)blocks * threads);
    uint64_t h[2 * kAcc];
    for (int i = 0; i < 2 * kAcc; ++i) h[i] = (0x0123456789abcdefull * (i + 1)) & ((1ull << 59) - 1);
    HE_CHECK_CUDA(ctx, cudaMemcpyAsync(in, h, sizeof(h), cudaMemcpyHostToDevice, ctx->stream));
    cudaEvent_t e0, e1;
    HE_CHECK_CUDA(ctx, cudaEventCreate(&e0));
    HE_CHECK_CUDA(ctx, cudaEventCreate(&e1));
    const double per = (double)blocks * threads * iters * kAcc;
    const int nv = n < 7 ? n : 7;
    for (int v = 0; v < nv; ++v) {
        auto launch = [&]() {
            ++ctx->launches;
            switch (v) {
                case 0: k_probe_chain<false><<<blocks, threads, 0, ctx->stream>>>(in, o, iters); break;
                case 6: k_probe_chain<true><<<blocks, threads, 0, ctx->stream>>>(in, o, iters); break;
                case 1: k_probe_cols<<<blocks, threads, 0, ctx->stream>>>(in, o, iters); break;
                case 2: k_probe_kara<<<blocks, threads, 0, ctx->stream>>>(in, o, iters); break;
                case 3: k_probe_op<0><<<blocks, threads, 0, ctx->stream>>>(in, o, iters); break;
                case 4: k_probe_op<1><<<blocks, threads, 0, ctx->stream>>>(in, o, iters); break;
                case 5: k_probe_op<2><<<blocks, threads, 0, ctx->stream>>>(in, o, iters); break;
                default: break;
            }
        };
        launch();
        launch();
        cudaEventRecord(e0, ctx->stream);
        for (int rep = 0; rep < 5; ++rep) launch();
        cudaEventRecord(e1, ctx->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        out[v] = per * 5 / (ms / 1e3);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return he_launch_check(ctx, "he_probe_int_ops");
}

extern "C" int he_probe_mem(he_ctx* ctx, double* out, int n) {
    if (!ctx || !out || n < 1) return HE_EINVAL;
    HE_NOT_RECORDING(ctx, "he_probe_mem");
    int sms = 0, dev = 0;
    HE_CHECK_CUDA(ctx, cudaGetDevice(&dev));
    HE_CHECK_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t sizes[2] = {(size_t)32 << 20, (size_t)2 << 30};   // bytes: L2-resident, HBM
    const int reps[2] = {40, 2};
    int rc = arena_reserve(ctx, sizes[1] / 8 + 64);
    if (rc) return rc;
    arena_reset(ctx);
    uint64_t* buf = arena_take(ctx, sizes[1] / 8);
    uint64_t* sink = arena_take(ctx, 8);
    HE_CHECK_CUDA(ctx, cudaMemsetAsync(buf, 1, sizes[1], ctx->stream));
    cudaEvent_t e0, e1;
    HE_CHECK_CUDA(ctx, cudaEventCreate(&e0));
    HE_CHECK_CUDA(ctx, cudaEventCreate(&e1));
    const int nv = n < 2 ? n : 2;
    for (int v = 0; v < nv; ++v) {
        const size_t n16 = sizes[v] / 16;
        k_probe_read<<<sms * 8, 256, 0, ctx->stream>>>((const uint4*)buf, n16, 1, sink);   // warm
        cudaEventRecord(e0, ctx->stream);
        k_probe_read<<<sms * 8, 256, 0, ctx->stream>>>((const uint4*)buf, n16, reps[v], sink);
        cudaEventRecord(e1, ctx->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        out[v] = (double)sizes[v] * reps[v] / (ms / 1e3) / 1e9;
        ctx->launches += 2;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return he_launch_check(ctx, "he_probe_mem");
}
