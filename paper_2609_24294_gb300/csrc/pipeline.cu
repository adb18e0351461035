// A transposition pipelined per piece: compression, all-to-all and
// decompression of successive pieces of one plan's messages overlap on three
// streams (paper Sec. III-E / V-B: the serial model is an upper bound because
// compression and communication could be pipelined per block).
//
// Piece k holds the messages whose destination peer d (0 .. P-1 within its
// communicator) has k = floor(d K / P), so every rank sends something in every
// piece, as a rank of a real machine would.  Stream A compresses piece k
// (fused pack, send layout), stream B moves it to the receive layout (the
// device-local stand-in for the exchange) once A has finished it, stream C
// decompresses and unpacks it once B has.  Events order the three streams;
// the caller's stream waits for the last piece.  The result is byte for byte
// that of the serial calls: every piece writes only its own messages' slots
// and boxes.
#include <algorithm>
#include <new>
#include <vector>

#include "zfpx_internal.h"

namespace zfpx {
namespace {

struct Piece {
    DevTable codec, chunks;         // 32-block units; 16-byte chunks of the permutation
    int nmsg = 0;
};

}  // namespace
}  // namespace zfpx

struct zfpx_pipeline_s {
    zfpx_plan_s *plan = nullptr;
    int rate = 0, dev = 0;
    std::vector<zfpx::Piece> pieces;
    cudaStream_t s[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t start = nullptr, end[3] = {nullptr, nullptr, nullptr};
    std::vector<cudaEvent_t> compressed, moved;
};

using namespace zfpx;

static void destroy_pipeline(zfpx_pipeline_s *pl)
{
    if (!pl) return;
    for (Piece &pc : pl->pieces) {
        cudaFree(pc.codec.d_msgs);
        cudaFree(pc.chunks.d_msgs);
    }
    for (cudaEvent_t e : pl->compressed) if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : pl->moved) if (e) cudaEventDestroy(e);
    if (pl->start) cudaEventDestroy(pl->start);
    for (cudaEvent_t e : pl->end) if (e) cudaEventDestroy(e);
    for (cudaStream_t st : pl->s) if (st) cudaStreamDestroy(st);
    delete pl;
}

extern "C" {

int zfpx_pipeline_create(zfpx_pipeline *out, zfpx_plan p, int rate, int pieces)
{
    if (!out || !p || !valid_codec_rate(rate) || pieces < 1) return ZFPX_EINVAL;
    *out = nullptr;
    // peers per communicator: the largest destination peer index + 1
    int P = 1;
    for (const HostMsg &m : p->msgs) P = std::max(P, m.dst_peer + 1);
    const int K = std::min(pieces, P);
    zfpx_pipeline_s *pl = new (std::nothrow) zfpx_pipeline_s;
    if (!pl) return ZFPX_ENOMEM;
    pl->plan = p;
    pl->rate = rate;
    if (cudaGetDevice(&pl->dev) != cudaSuccess) { delete pl; return ZFPX_ECUDA; }
    pl->pieces.resize(K);
    int rc = ZFPX_OK;
    for (int k = 0; k < K && !rc; k++) {
        std::vector<int> subset;
        for (size_t i = 0; i < p->msgs.size(); i++)
            if ((int64_t)p->msgs[i].dst_peer * K / P == k) subset.push_back((int)i);
        Piece &pc = pl->pieces[k];
        pc.nmsg = (int)subset.size();
        if (subset.empty()) continue;
        std::vector<MsgDev> h;
        int64_t u = host_table(p, rate, UNIT_BLOCKS32, subset, h);
        rc = upload_table(h, u, &pc.codec);
        if (!rc) {
            u = host_table(p, rate, UNIT_CHUNK16, subset, h);
            rc = upload_table(h, u, &pc.chunks);
        }
    }
    for (int i = 0; i < 3 && !rc; i++)
        if (cudaStreamCreateWithFlags(&pl->s[i], cudaStreamNonBlocking) != cudaSuccess) rc = ZFPX_ECUDA;
    if (!rc && cudaEventCreateWithFlags(&pl->start, cudaEventDisableTiming) != cudaSuccess) rc = ZFPX_ECUDA;
    for (int i = 0; i < 3 && !rc; i++)
        if (cudaEventCreateWithFlags(&pl->end[i], cudaEventDisableTiming) != cudaSuccess) rc = ZFPX_ECUDA;
    pl->compressed.assign(K, nullptr);
    pl->moved.assign(K, nullptr);
    for (int k = 0; k < K && !rc; k++)
        if (cudaEventCreateWithFlags(&pl->compressed[k], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&pl->moved[k], cudaEventDisableTiming) != cudaSuccess)
            rc = ZFPX_ECUDA;
    if (rc) {
        destroy_pipeline(pl);
        return rc;
    }
    *out = pl;
    return ZFPX_OK;
}

int zfpx_pipeline_pieces(zfpx_pipeline pl) { return pl ? (int)pl->pieces.size() : ZFPX_EINVAL; }

int zfpx_pipeline_run(zfpx_pipeline pl, const float *d_src, uint8_t *d_send, uint8_t *d_recv, size_t buf_bytes,
                      float *d_dst, void *stream)
{
    if (!pl || !d_src || !d_send || !d_recv || !d_dst) return ZFPX_EINVAL;
    zfpx_plan_s *p = pl->plan;
    const int64_t need = buffer_bytes(p, pl->rate);
    if ((int64_t)buf_bytes < need) return ZFPX_ESIZE;
    if (((uintptr_t)d_send & 15u) || ((uintptr_t)d_recv & 15u)) return ZFPX_EINVAL;
    if (d_send < d_recv + need && d_recv < d_send + need) return ZFPX_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ZFPX_ECUDA;
    if (dev != pl->dev) return ZFPX_EINVAL;
    cudaStream_t caller = (cudaStream_t)stream;
    if (cudaEventRecord(pl->start, caller) != cudaSuccess) return ZFPX_ECUDA;
    for (cudaStream_t st : pl->s)
        if (cudaStreamWaitEvent(st, pl->start, 0) != cudaSuccess) return ZFPX_ECUDA;
    const int vec_src = codec_vec_ok(d_src, p->ss, p) ? 1 : 0;
    const int vec_dst = codec_vec_ok(d_dst, p->ds, p) ? 1 : 0;
    for (size_t k = 0; k < pl->pieces.size(); k++) {
        const Piece &pc = pl->pieces[k];
        LaunchGeom g{};
        g.nmsg = pc.nmsg;
        for (int a = 0; a < 3; a++) { g.ss[a] = p->ss[a]; g.ds[a] = p->ds[a]; }
        int rc = ZFPX_OK;
        if (pc.nmsg) {
            g.msgs = pc.codec.d_msgs;
            g.nunits = pc.codec.nunits;
            rc = launch_encode(p->dims, pl->rate, d_src, d_send, g, ZFPX_LAYOUT_SEND, vec_src, pl->s[0]);
        }
        if (rc) return rc;
        if (cudaEventRecord(pl->compressed[k], pl->s[0]) != cudaSuccess ||
            cudaStreamWaitEvent(pl->s[1], pl->compressed[k], 0) != cudaSuccess)
            return ZFPX_ECUDA;
        if (pc.nmsg) {
            g.msgs = pc.chunks.d_msgs;
            g.nunits = pc.chunks.nunits;
            rc = launch_permute(d_send, d_recv, g, pl->rate, p->dims, pl->s[1]);
        }
        if (rc) return rc;
        if (cudaEventRecord(pl->moved[k], pl->s[1]) != cudaSuccess ||
            cudaStreamWaitEvent(pl->s[2], pl->moved[k], 0) != cudaSuccess)
            return ZFPX_ECUDA;
        if (pc.nmsg) {
            g.msgs = pc.codec.d_msgs;
            g.nunits = pc.codec.nunits;
            rc = launch_decode(p->dims, pl->rate, d_recv, d_dst, g, ZFPX_LAYOUT_RECV, vec_dst, pl->s[2]);
        }
        if (rc) return rc;
    }
    // the caller's stream joins all three (stream C's last piece already follows
    // every earlier launch; joining each stream also closes a stream capture)
    for (int i = 0; i < 3; i++)
        if (cudaEventRecord(pl->end[i], pl->s[i]) != cudaSuccess || cudaStreamWaitEvent(caller, pl->end[i], 0) != cudaSuccess)
            return ZFPX_ECUDA;
    return ZFPX_OK;
}

void zfpx_pipeline_destroy(zfpx_pipeline pl) { destroy_pipeline(pl); }

}  // extern "C"
