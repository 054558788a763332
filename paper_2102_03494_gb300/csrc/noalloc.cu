// noalloc.cu -- he_rotate_noalloc: the plain rotation without any device allocation.
//
// Some callers cannot allocate device memory when they rotate: a process whose device memory
// is already handed out by another allocator (a framework's caching pool that reserved the
// GPU), a serving loop that must not pay for, or synchronise on, cudaMalloc/cudaFree in its
// request path, or host code running where the CUDA allocator may not be called.  For them
// this entry point takes its key-switching scratch from one file-scope device array whose
// size is fixed when the library is built, instead of from the context's growable scratch.
//
// The array lives in every GPU that loads the library, until the process exits.  Each call
// overwrites it completely before reading it (the input copy, ModUp digits, inner products
// and ModDown values are all written first), so nothing has to be cleared between calls.
// All calls share it: two calls that overlap on the GPU (two streams, two contexts, two host
// threads) race on it and must be serialised by the caller.
#include <mutex>
#include <vector>

#include "eval.cuh"
#include "kernels.cuh"

#define HE_NOALLOC_SCRATCH_BYTES (16ull << 20)

static __device__ __align__(256) uint64_t g_noalloc_scratch[HE_NOALLOC_SCRATCH_BYTES / 8];

// Device address of g_noalloc_scratch on the current device.  In host code the symbol is
// only a host-side stand-in, so the address is looked up once per device (with that device
// current) and cached.  The first call on a device does this set-up; make that first call
// before any stream capture.
static int noalloc_scratch(he_ctx* ctx, uint64_t** out) {
    static std::mutex mu;
    static std::vector<uint64_t*> by_device;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return he_fail(ctx, HE_ECUDA, cudaGetErrorString(e));
    std::lock_guard<std::mutex> lock(mu);
    if ((int)by_device.size() <= dev) by_device.resize(dev + 1, nullptr);
    if (!by_device[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return he_fail(ctx, HE_ECUDA, std::string("he_rotate_noalloc: cudaGetSymbolAddress: ") +
                                              cudaGetErrorString(e));
        by_device[dev] = (uint64_t*)p;
    }
    *out = by_device[dev];
    return HE_OK;
}

static size_t align_words(size_t n) { return (n + 31) & ~(size_t)31; }   // 256-byte slices

extern "C" int he_rotate_noalloc(he_ctx* ctx, const he_ct* in, int32_t step, he_ct* out) {
    if (!ctx) return HE_EINVAL;
    // while a graph is recorded the pointer tables below would go to buffers the graph
    // allocates, and a replay would share the static array with later calls: refused
    HE_NOT_RECORDING(ctx, "he_rotate_noalloc");
    int rc = check_ct(ctx, in, ctx->L, HE_NTT, "he_rotate_noalloc input");
    if (!rc) rc = check_ct(ctx, out, ctx->L, -1, "he_rotate_noalloc output");
    if (rc) return rc;
    const uint32_t g = galois_elt(ctx, step);
    const uint64_t* key = nullptr;
    if ((rc = he_get_key(ctx, g, &key))) return rc;
    const size_t N = ctx->N, L = ctx->L, LK = ctx->L + ctx->K;
    const size_t w_x = align_words(2 * L * N), w_t = align_words(L * N),
                 w_d = align_words(ctx->dnum * LK * N), w_u = align_words(2 * LK * N),
                 w_v = align_words(2 * L * N);
    const size_t need = (w_x + w_t + w_d + w_u + w_v) * 8;
    if (need > HE_NOALLOC_SCRATCH_BYTES)
        return he_fail(ctx, HE_EINVAL, "he_rotate_noalloc: these parameters need " +
                                           std::to_string(need) + " bytes of scratch, more than the " +
                                           std::to_string(HE_NOALLOC_SCRATCH_BYTES) + " built in");
    uint64_t* base = nullptr;
    if ((rc = noalloc_scratch(ctx, &base))) return rc;
    uint64_t* X = base;
    RotBufs b;
    b.T = X + w_x;
    b.D = b.T + w_t;
    b.u = b.D + w_d;
    b.v = b.u + w_u;
    // copy the input first so that `in` and `out` may alias
    HE_CHECK_CUDA(ctx, cudaMemcpyAsync(X, in->data, 2 * L * N * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    const uint64_t* c0 = X;
    uint64_t* o = out->data;
    auto c0p = upload_ptrs(ctx, {c0});
    auto op = upload_out_ptrs(ctx, {o});
    if (!c0p || !op) return he_fail(ctx, HE_ECUDA, "he_rotate_noalloc: pointer table upload failed");
    modup_items(ctx, X, 1, g, b);
    ks_items(ctx, 1, key, 1u, g, c0p, nullptr, op, b);
    out->domain = HE_NTT;
    ctx->ops[2] += 1;
    ctx->ops[3] += 1;
    return he_launch_check(ctx, "he_rotate_noalloc");
}
