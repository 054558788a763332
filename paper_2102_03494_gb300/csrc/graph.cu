// graph.cu -- recorded call sequences: library calls captured once into a CUDA graph and
// replayed with one submission.
//
// he_graph_begin switches the context's work onto a private non-blocking stream in relaxed
// capture mode; the library calls that follow run their ordinary host code and their kernels
// and copies are recorded, not executed, until he_graph_end instantiates the graph.  What
// keeps the recording valid for later replays:
//   * scratch: the context's arena at its current generation (shared), or a copy of its size
//     that the graph owns; while recording, neither the arena nor the network buffer may grow
//     (a call that would need it fails), so the calls must have run once before;
//   * pointer tables, weights and other call arguments go into device buffers the graph owns
//     (upload_small / upload_host check ctx->rec) instead of the reused staging ring or host
//     memory that belongs to the recorded call;
//   * phase timing is off, and the launch / operation counters are rolled back (a replay adds
//     what the recording counted).
// A replay checks that nothing it points to has gone: the layer plans it used, the resident
// keys (dropped keys bump keys_epoch), the shared arena and the network buffer generations.
#include <algorithm>

#include "he_internal.cuh"

void graph_release(he_ctx::LayerGraph& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    if (g.arena.base) cudaFree(g.arena.base);
    for (void* p : g.allocs) cudaFree(p);
    g = he_ctx::LayerGraph{};
}

// own = 0: record on the context's scratch.  own = 1: on a fresh arena of the context's
// current capacity.  own = 2: on the arena the context holds now (the caller saved the user's
// in *adopt_saved); either of the last two is the graph's afterwards.
static int begin_recording(he_ctx* ctx, int own, const Arena* adopt_saved) {
    if (ctx->rec) return he_fail(ctx, HE_EINVAL, "he_graph_begin: already recording");
    HE_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    auto* r = new he_ctx::Recording();
    r->g.keys_epoch = ctx->keys_epoch;
    r->g.shared = own == 0;
    r->user_stream = ctx->stream;
    r->saved = adopt_saved ? *adopt_saved : ctx->arena;
    r->timing = ctx->timing;
    r->launches0 = ctx->launches;
    for (int i = 0; i < 4; ++i) r->ops0[i] = ctx->ops[i];
    if (own == 1) {
        Arena fresh;
        if (ctx->arena.cap && cudaMalloc(&fresh.base, ctx->arena.cap) != cudaSuccess) {
            cudaGetLastError();
            delete r;
            return he_fail(ctx, HE_ENOMEM, "he_graph_begin: scratch allocation failed");
        }
        fresh.cap = ctx->arena.cap;
        ctx->arena = fresh;
    }
    r->g.arena_epoch = ctx->arena_epoch;
    r->g.net_epoch = ctx->net_epoch;
    r->g.pk_epoch = ctx->pk_epoch;
    // on failure below only the fresh arena of own == 1 is undone; otherwise the context's
    // arena is left as it is (the caller of own == 2 still holds its saved one)
    if (cudaStreamCreateWithFlags(&r->cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        if (own == 1) {
            if (ctx->arena.base) cudaFree(ctx->arena.base);
            ctx->arena = r->saved;
        }
        delete r;
        return he_fail(ctx, HE_ECUDA, "he_graph_begin: stream creation failed");
    }
    const cudaError_t e = cudaStreamBeginCapture(r->cs, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaStreamDestroy(r->cs);
        if (own == 1) {
            if (ctx->arena.base) cudaFree(ctx->arena.base);
            ctx->arena = r->saved;
        }
        delete r;
        return he_fail(ctx, HE_ECUDA, std::string("he_graph_begin: ") + cudaGetErrorString(e));
    }
    ctx->stream = r->cs;
    ctx->timing = false;
    ctx->rec = r;
    return HE_OK;
}

// Ends the recording; `failed` (a call inside it failed) discards the graph.
static int end_recording(he_ctx* ctx, int failed, int32_t* graph_out) {
    he_ctx::Recording* r = ctx->rec;
    if (!r) return he_fail(ctx, HE_EINVAL, "he_graph_end: not recording");
    he_ctx::LayerGraph g = std::move(r->g);
    const int spoiled = r->failed;
    cudaError_t e = cudaStreamEndCapture(r->cs, &g.graph);
    int rc = failed;
    if (!rc && spoiled)
        rc = he_fail(ctx, spoiled, "he_graph_end: a call failed while recording (" + ctx->err +
                                       "); the recording is discarded");
    if (!rc && e != cudaSuccess)
        rc = he_fail(ctx, HE_ECUDA, std::string("he_graph_end: ") + cudaGetErrorString(e));
    if (!rc && ctx->arena_epoch != g.arena_epoch)       // growth is refused while recording
        rc = he_fail(ctx, HE_ECUDA, "he_graph_end: scratch changed while recording");
    if (!rc && (e = cudaGraphInstantiate(&g.exec, g.graph, 0)) != cudaSuccess)
        rc = he_fail(ctx, HE_ECUDA, std::string("he_graph_end: ") + cudaGetErrorString(e));
    cudaGetLastError();
    g.launches = ctx->launches - r->launches0;
    for (int i = 0; i < 4; ++i) g.ops[i] = ctx->ops[i] - r->ops0[i];
    ctx->launches = r->launches0;                        // the recording executed nothing
    for (int i = 0; i < 4; ++i) ctx->ops[i] = r->ops0[i];
    if (!g.shared) {
        g.arena = ctx->arena;
        g.arena.used = 0;
        ctx->arena = r->saved;
    }
    ctx->stream = r->user_stream;
    ctx->timing = r->timing;
    cudaStreamDestroy(r->cs);
    ctx->rec = nullptr;
    delete r;
    std::sort(g.plans.begin(), g.plans.end());
    g.plans.erase(std::unique(g.plans.begin(), g.plans.end()), g.plans.end());
    if (rc) {
        graph_release(g);
        return rc;
    }
    const int32_t id = ctx->next_graph++;
    ctx->graphs[id] = std::move(g);
    if (graph_out) *graph_out = id;
    return HE_OK;
}

void recording_abort(he_ctx* ctx) {
    if (ctx->rec) end_recording(ctx, HE_EINVAL, nullptr);
}

extern "C" int he_graph_begin(he_ctx* ctx, int share_scratch) {
    if (!ctx) return HE_EINVAL;
    return begin_recording(ctx, share_scratch ? 0 : 1, nullptr);
}

extern "C" int he_graph_end(he_ctx* ctx, int32_t* graph_out) {
    if (!ctx) return HE_EINVAL;
    if (!graph_out) {
        if (ctx->rec) end_recording(ctx, HE_EINVAL, nullptr);
        return he_fail(ctx, HE_EINVAL, "he_graph_end: null argument");
    }
    return end_recording(ctx, HE_OK, graph_out);
}

extern "C" int he_ffconv_graph_create(he_ctx* ctx, int32_t plan, const he_ct* ct_in, int B,
                                      he_ct* ct_out, int share_scratch, int32_t* graph_out) {
    if (!ctx) return HE_EINVAL;
    if (!ct_in || !ct_out || !graph_out || B < 1)
        return he_fail(ctx, HE_EINVAL, "he_ffconv_graph_create: null argument");
    if (ctx->rec) return he_fail(ctx, HE_EINVAL, "he_ffconv_graph_create: already recording");
    if (ctx->plans.find(plan) == ctx->plans.end())
        return he_fail(ctx, HE_EINVAL, "he_ffconv_graph_create: no such plan");
    const bool timing = ctx->timing;
    ctx->timing = false;
    // the uncaptured run sizes the scratch (for an own scratch: a fresh arena of exactly this
    // call's size), sets kernel attributes and leaves the result in ct_out
    // (the fresh arena is not the context's: its generation counter is put back afterwards,
    // so graphs recorded on the context's own scratch stay valid)
    const Arena saved = ctx->arena;
    const uint64_t epoch0 = ctx->arena_epoch;
    if (!share_scratch) ctx->arena = Arena{};
    int rc = he_ffconv_layer_planned(ctx, plan, ct_in, B, ct_out);
    if (!rc) rc = check_device_error(ctx);
    ctx->timing = timing;
    if (!rc) rc = begin_recording(ctx, share_scratch ? 0 : 2, &saved);
    else if (!share_scratch) cudaStreamSynchronize(ctx->stream);
    if (rc) {
        if (!share_scratch) {
            if (ctx->arena.base) cudaFree(ctx->arena.base);
            ctx->arena = saved;
            ctx->arena_epoch = epoch0;
        }
        return rc;
    }
    rc = he_ffconv_layer_planned(ctx, plan, ct_in, B, ct_out);
    rc = end_recording(ctx, rc, graph_out);
    if (!share_scratch) ctx->arena_epoch = epoch0;
    return rc;
}

extern "C" int he_graph_launch(he_ctx* ctx, int32_t graph) {
    if (!ctx) return HE_EINVAL;
    if (ctx->rec) return he_fail(ctx, HE_EINVAL, "he_graph_launch: recording in progress");
    auto it = ctx->graphs.find(graph);
    if (it == ctx->graphs.end()) return he_fail(ctx, HE_EINVAL, "he_graph_launch: no such graph");
    const he_ctx::LayerGraph& g = it->second;
    for (int32_t p : g.plans)
        if (ctx->plans.find(p) == ctx->plans.end())
            return he_fail(ctx, HE_EINVAL, "he_graph_launch: a layer plan the graph uses was freed");
    if (g.keys_epoch != ctx->keys_epoch)
        return he_fail(ctx, HE_EINVAL, "he_graph_launch: resident keys were dropped since recording");
    if (g.shared && g.arena_epoch != ctx->arena_epoch)
        return he_fail(ctx, HE_EINVAL, "he_graph_launch: the context scratch was reallocated since recording");
    if (g.net_epoch != ctx->net_epoch)
        return he_fail(ctx, HE_EINVAL, "he_graph_launch: the network buffer was reallocated since recording");
    if (g.pk_epoch != ctx->pk_epoch)
        return he_fail(ctx, HE_EINVAL, "he_graph_launch: the tap product buffer was reallocated since recording");
    HE_CHECK_CUDA(ctx, cudaGraphLaunch(g.exec, ctx->stream));
    ctx->launches += g.launches;
    for (int i = 0; i < 4; ++i) ctx->ops[i] += g.ops[i];
    return HE_OK;
}

extern "C" int he_graph_free(he_ctx* ctx, int32_t graph) {
    if (!ctx) return HE_EINVAL;
    HE_NOT_RECORDING(ctx, "he_graph_free");
    auto it = ctx->graphs.find(graph);
    if (it == ctx->graphs.end()) return he_fail(ctx, HE_EINVAL, "he_graph_free: no such graph");
    cudaStreamSynchronize(ctx->stream);
    graph_release(it->second);
    ctx->graphs.erase(it);
    return HE_OK;
}
