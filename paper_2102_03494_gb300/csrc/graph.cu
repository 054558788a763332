// graph.cu -- captured layers: a planned FFConv layer recorded once into a CUDA graph and
// replayed with one submission.
//
// The capture runs the ordinary host path of he_ffconv_layer_planned on a private
// non-blocking stream in relaxed capture mode.  Three things make the recorded work valid
// for later replays: the scratch arena is the graph's own (sized by one uncaptured run of
// the same call just before) or the context's at a recorded generation (launches check it),
// pointer tables and weights are uploaded into device buffers the graph owns (upload_small
// checks ctx->capture_allocs) rather than into the reused staging ring, and phase timing is
// off while recording.
#include "he_internal.cuh"

void graph_release(he_ctx::LayerGraph& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    if (g.arena.base) cudaFree(g.arena.base);
    for (void* p : g.allocs) cudaFree(p);
    g = he_ctx::LayerGraph{};
}

extern "C" int he_ffconv_graph_create(he_ctx* ctx, int32_t plan, const he_ct* ct_in, int B,
                                      he_ct* ct_out, int share_scratch, int32_t* graph_out) {
    if (!ctx) return HE_EINVAL;
    if (!ct_in || !ct_out || !graph_out || B < 1)
        return he_fail(ctx, HE_EINVAL, "he_ffconv_graph_create: null argument");
    if (ctx->plans.find(plan) == ctx->plans.end())
        return he_fail(ctx, HE_EINVAL, "he_ffconv_graph_create: no such plan");
    he_ctx::LayerGraph g;
    g.plan = plan;
    g.keys_epoch = ctx->keys_epoch;
    g.shared = share_scratch != 0;
    const Arena saved = ctx->arena;
    const bool timing = ctx->timing;
    if (!g.shared) ctx->arena = Arena{};
    ctx->timing = false;
    // the uncaptured run: sizes the graph's arena, sets kernel attributes, fills ct_out
    int rc = he_ffconv_layer_planned(ctx, plan, ct_in, B, ct_out);
    if (!rc) rc = check_device_error(ctx);
    g.arena_epoch = ctx->arena_epoch;
    const uint64_t launches1 = ctx->launches;
    uint64_t ops1[4];
    for (int i = 0; i < 4; ++i) ops1[i] = ctx->ops[i];
    cudaStream_t user = ctx->stream, cs = nullptr;
    if (!rc && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        rc = he_fail(ctx, HE_ECUDA, "he_ffconv_graph_create: stream creation failed");
    }
    if (!rc) {
        ctx->stream = cs;
        ctx->capture_allocs = &g.allocs;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) {
            rc = he_fail(ctx, HE_ECUDA, std::string("he_ffconv_graph_create: ") + cudaGetErrorString(e));
        } else {
            rc = he_ffconv_layer_planned(ctx, plan, ct_in, B, ct_out);
            e = cudaStreamEndCapture(cs, &g.graph);
            if (!rc && ctx->arena_epoch != g.arena_epoch)   // cannot happen: same call, same sizes
                rc = he_fail(ctx, HE_ECUDA, "he_ffconv_graph_create: scratch grew while capturing");
            if (!rc && e != cudaSuccess)
                rc = he_fail(ctx, HE_ECUDA, std::string("he_ffconv_graph_create: ") + cudaGetErrorString(e));
            if (!rc && (e = cudaGraphInstantiate(&g.exec, g.graph, 0)) != cudaSuccess)
                rc = he_fail(ctx, HE_ECUDA, std::string("he_ffconv_graph_create: ") + cudaGetErrorString(e));
        }
        cudaGetLastError();
        ctx->stream = user;
        ctx->capture_allocs = nullptr;
    }
    g.launches = ctx->launches - launches1;
    for (int i = 0; i < 4; ++i) g.ops[i] = ctx->ops[i] - ops1[i];
    // the recording executed nothing: count only the uncaptured run
    ctx->launches = launches1;
    for (int i = 0; i < 4; ++i) ctx->ops[i] = ops1[i];
    if (!g.shared) {
        g.arena = ctx->arena;
        g.arena.used = 0;
        ctx->arena = saved;
    }
    ctx->timing = timing;
    if (cs) cudaStreamDestroy(cs);
    if (rc) {
        graph_release(g);
        return rc;
    }
    const int32_t id = ctx->next_graph++;
    ctx->graphs[id] = g;
    *graph_out = id;
    return HE_OK;
}

extern "C" int he_graph_launch(he_ctx* ctx, int32_t graph) {
    if (!ctx) return HE_EINVAL;
    auto it = ctx->graphs.find(graph);
    if (it == ctx->graphs.end()) return he_fail(ctx, HE_EINVAL, "he_graph_launch: no such graph");
    const he_ctx::LayerGraph& g = it->second;
    if (ctx->plans.find(g.plan) == ctx->plans.end())
        return he_fail(ctx, HE_EINVAL, "he_graph_launch: the graph's plan was freed");
    if (g.keys_epoch != ctx->keys_epoch)
        return he_fail(ctx, HE_EINVAL, "he_graph_launch: resident keys were dropped since capture");
    if (g.shared && g.arena_epoch != ctx->arena_epoch)
        return he_fail(ctx, HE_EINVAL, "he_graph_launch: the context scratch was reallocated since capture");
    HE_CHECK_CUDA(ctx, cudaGraphLaunch(g.exec, ctx->stream));
    ctx->launches += g.launches;
    for (int i = 0; i < 4; ++i) ctx->ops[i] += g.ops[i];
    return HE_OK;
}

extern "C" int he_graph_free(he_ctx* ctx, int32_t graph) {
    if (!ctx) return HE_EINVAL;
    auto it = ctx->graphs.find(graph);
    if (it == ctx->graphs.end()) return he_fail(ctx, HE_EINVAL, "he_graph_free: no such graph");
    cudaStreamSynchronize(ctx->stream);
    graph_release(it->second);
    ctx->graphs.erase(it);
    return HE_OK;
}
