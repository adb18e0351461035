// The full transposition pair (paper Sec. II-B: z -> lambda by rows, then
// lambda -> theta by columns; Sec. VI notes the second is built like the
// first) as one CUDA graph: pack+compress, the device-local all-to-all and
// decompress+unpack for each of the two plans, six launches replayed with a
// single graph launch.
#include <new>

#include "zfpx_internal.h"

struct zfpx_graph_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
};

using namespace zfpx;

extern "C" {

int zfpx_pair_graph_create(zfpx_graph *out, zfpx_plan first, zfpx_plan second, int rate, const float *d_src,
                           float *d_mid, float *d_dst, uint8_t *d_send, uint8_t *d_recv, size_t buf_bytes,
                           int fold_permute)
{
    if (!out) return ZFPX_EINVAL;
    *out = nullptr;
    if (!first || !second || !d_src || !d_mid || !d_dst || !d_send || !d_recv) return ZFPX_EINVAL;
    if (!valid_codec_rate(rate)) return ZFPX_EINVAL;
    if (first->n[0] != second->n[0] || first->n[1] != second->n[1] || first->n[2] != second->n[2])
        return ZFPX_EINVAL;
    const int64_t need = buffer_bytes(first, rate) > buffer_bytes(second, rate) ? buffer_bytes(first, rate)
                                                                                 : buffer_bytes(second, rate);
    if ((int64_t)buf_bytes < need) return ZFPX_ESIZE;
    // device tables must exist before capture (no allocation while capturing)
    int rc = zfpx_plan_prepare(first, rate);
    if (!rc) rc = zfpx_plan_prepare(second, rate);
    if (rc) return rc;

    zfpx_graph_s *g = new (std::nothrow) zfpx_graph_s;
    if (!g) return ZFPX_ENOMEM;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { delete g; return ZFPX_ECUDA; }
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaStreamDestroy(st);
        delete g;
        return ZFPX_ECUDA;
    }
    const uint64_t before = zfpx_launch_count();
    const zfpx_plan plans[2] = {first, second};
    const float *srcs[2] = {d_src, d_mid};
    float *dsts[2] = {d_mid, d_dst};
    for (int s = 0; s < 2 && !rc; s++) {
        const size_t len = (size_t)buffer_bytes(plans[s], rate);
        if (fold_permute) {
            rc = zfpx_pack_compress(plans[s], rate, srcs[s], d_recv, len, ZFPX_LAYOUT_RECV, st);
        } else {
            rc = zfpx_pack_compress(plans[s], rate, srcs[s], d_send, len, ZFPX_LAYOUT_SEND, st);
            if (!rc) rc = zfpx_permute(plans[s], rate, d_send, d_recv, len, st);
        }
        if (!rc) rc = zfpx_decompress_unpack(plans[s], rate, d_recv, len, dsts[s], ZFPX_LAYOUT_RECV, st);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(st, &graph);
    cudaStreamDestroy(st);
    if (rc || ec != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        delete g;
        return rc ? rc : ZFPX_ECUDA;
    }
    if (cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) {
        cudaGraphDestroy(graph);
        delete g;
        return ZFPX_ECUDA;
    }
    g->graph = graph;
    g->launches = (int)(zfpx_launch_count() - before);
    uncount_launches((uint64_t)g->launches);             // recorded, not run
    *out = g;
    return ZFPX_OK;
}

// Generic capture: launches are counted when the graph is launched, not
// when they are recorded.
static thread_local uint64_t g_capture_start = 0;

int zfpx_capture_begin(void *stream)
{
    if (!stream) return ZFPX_EINVAL;
    if (cudaStreamBeginCapture((cudaStream_t)stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return ZFPX_ECUDA;
    g_capture_start = zfpx_launch_count();
    return ZFPX_OK;
}

int zfpx_capture_end(zfpx_graph *out, void *stream)
{
    if (!out || !stream) return ZFPX_EINVAL;
    *out = nullptr;
    cudaGraph_t graph = nullptr;
    if (cudaStreamEndCapture((cudaStream_t)stream, &graph) != cudaSuccess || !graph) return ZFPX_ECUDA;
    zfpx_graph_s *g = new (std::nothrow) zfpx_graph_s;
    if (!g) { cudaGraphDestroy(graph); return ZFPX_ENOMEM; }
    if (cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) {
        cudaGraphDestroy(graph);
        delete g;
        return ZFPX_ECUDA;
    }
    g->graph = graph;
    g->launches = (int)(zfpx_launch_count() - g_capture_start);
    uncount_launches((uint64_t)g->launches);
    *out = g;
    return ZFPX_OK;
}

int zfpx_graph_launch(zfpx_graph g, void *stream)
{
    if (!g || !g->exec) return ZFPX_EINVAL;
    if (cudaGraphLaunch(g->exec, (cudaStream_t)stream) != cudaSuccess) return ZFPX_ECUDA;
    for (int i = 0; i < g->launches; i++) count_launch();
    return ZFPX_OK;
}

int zfpx_graph_num_kernels(zfpx_graph g) { return g ? g->launches : ZFPX_EINVAL; }

void zfpx_graph_destroy(zfpx_graph g)
{
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

}  // extern "C"
