// Pencil-transposition plan: message boxes, block counts, fixed byte offsets
// and the device tables the kernels read (paper Sec. II-B; Table 1).
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <new>

#include "zfpx_internal.h"

namespace zfpx {

static std::atomic<uint64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void uncount_launches(uint64_t n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }

bool valid_codec_rate(int rate) { return rate == 8 || rate == 16; }

static bool valid_rate(int rate) { return rate == ZFPX_RATE_F32 || rate == ZFPX_RATE_F16 || valid_codec_rate(rate); }

int num_sms()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

int occupancy(const void *fn, int threads)
{
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> cache;
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_pair(fn, threads);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, 0) != cudaSuccess || n < 1) n = 1;
    cache[key] = n;
    return n;
}

int check_launch()
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ZFPX_OK : ZFPX_ECUDA;
}

static const int64_t kAlign = 256;
static int64_t align_up(int64_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
static int64_t ceil4(int64_t v) { return (v + 3) / 4; }

// Largest extent per axis: a block's origin plus 4 (the kernels test x0 + 4 <=
// n in 32-bit arithmetic) stays below 2^31.
constexpr int64_t kMaxExtent = ((int64_t)1 << 31) - 8;
// Most messages a plan may hold (P p_c for z -> lambda, P p_r for lambda ->
// theta): 2^24 descriptors, about 1.3 GB of host tables.
constexpr int64_t kMaxMessages = (int64_t)1 << 24;

static void block_counts(int dims, const HostMsg &m, int64_t b[3])
{
    b[0] = ceil4(m.nx);
    if (dims == 3) { b[1] = ceil4(m.ny); b[2] = ceil4(m.nz); }
    else if (dims == 2) { b[1] = ceil4(m.ny); b[2] = m.nz; }
    else { b[1] = m.ny; b[2] = m.nz; }
}

int64_t message_bytes(const zfpx_plan_s *p, const HostMsg &m, int rate)
{
    const int64_t nv = m.nx * m.ny * m.nz;
    if (rate == ZFPX_RATE_F32) return 4 * nv;
    if (rate == ZFPX_RATE_F16) return 2 * nv;
    int64_t b[3];
    block_counts(p->dims, m, b);
    const int64_t nb = b[0] * b[1] * b[2];
    return p->dims == 3 ? nb * 8 * rate : p->dims == 2 ? nb * 2 * rate : nb * rate / 2;
}

// Offsets of every message (send order index) in the given layout.
std::vector<int64_t> layout_offsets(const zfpx_plan_s *p, int rate, int layout, int64_t *total)
{
    const size_t M = p->msgs.size();
    std::vector<size_t> order(M);
    for (size_t i = 0; i < M; i++) order[i] = i;
    if (layout == ZFPX_LAYOUT_RECV) {
        std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
            const HostMsg &x = p->msgs[a], &y = p->msgs[b];
            if (x.dst != y.dst) return x.dst < y.dst;
            return x.src_peer < y.src_peer;
        });
    }
    std::vector<int64_t> off(M, 0);
    int64_t o = 0;
    for (size_t i : order) {
        off[i] = o;
        o = align_up(o + message_bytes(p, p->msgs[i], rate));
    }
    if (total) *total = o;
    return off;
}

int64_t buffer_bytes(const zfpx_plan_s *p, int rate)
{
    int64_t t = 0;
    layout_offsets(p, rate, ZFPX_LAYOUT_SEND, &t);
    return t;
}

static void split(int64_t extent, int parts, int mode, std::vector<int64_t> &start, std::vector<int64_t> &len)
{
    start.resize(parts);
    len.resize(parts);
    if (mode == ZFPX_SPLIT_TABLE1) {
        for (int i = 0; i < parts; i++) { len[i] = extent / parts; start[i] = i * len[i]; }
        return;
    }
    int64_t base = extent / parts, rem = extent % parts, s = 0;
    for (int i = 0; i < parts; i++) {
        len[i] = base + (i < rem ? 1 : 0);
        start[i] = s;
        s += len[i];
    }
}

int64_t host_table(const zfpx_plan_s *p, int rate, UnitKind kind, const std::vector<int> &subset,
                   std::vector<MsgDev> &h)
{
    const size_t M = p->msgs.size();
    const std::vector<int64_t> so = layout_offsets(p, rate, ZFPX_LAYOUT_SEND, nullptr);
    const std::vector<int64_t> ro = layout_offsets(p, rate, ZFPX_LAYOUT_RECV, nullptr);
    const size_t n = subset.empty() ? M : subset.size();
    h.assign(n, MsgDev{});
    int64_t units = 0;
    for (size_t j = 0; j < n; j++) {
        const size_t i = subset.empty() ? j : (size_t)subset[j];
        const HostMsg &m = p->msgs[i];
        MsgDev &d = h[j];
        int64_t b[3];
        block_counts(p->dims, m, b);
        d.src_off = m.x0 * p->ss[0] + m.y0 * p->ss[1] + m.z0 * p->ss[2];
        d.dst_off = m.x0 * p->ds[0] + m.y0 * p->ds[1] + m.z0 * p->ds[2];
        d.off[0] = so[i];
        d.off[1] = ro[i];
        d.nx = (int32_t)m.nx; d.ny = (int32_t)m.ny; d.nz = (int32_t)m.nz;
        d.bx = (int32_t)b[0]; d.by = (int32_t)b[1]; d.bz = (int32_t)b[2];
        d.nblocks = b[0] * b[1] * b[2];
        set_block_divisors(d);
        d.unit0 = units;
        if (kind == UNIT_BLOCKS32) units += (d.nblocks + 31) / 32;
        else if (kind == UNIT_QUADS) units += ceil4(m.nx) * m.ny * m.nz;
        else units += (message_bytes(p, m, rate) + 15) / 16;
    }
    return units;
}

int upload_table(const std::vector<MsgDev> &h, int64_t units, DevTable *t)
{
    t->d_msgs = nullptr;
    t->nunits = units;
    if (h.empty()) return ZFPX_OK;
    const size_t tb = (h.size() * sizeof(MsgDev) + 255) / 256 * 256;
    if (cudaMalloc((void **)&t->d_msgs, tb) != cudaSuccess) return ZFPX_ENOMEM;
    if (cudaMemcpy(t->d_msgs, h.data(), h.size() * sizeof(MsgDev), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(t->d_msgs);
        t->d_msgs = nullptr;
        return ZFPX_ECUDA;
    }
    return ZFPX_OK;
}

int get_table(zfpx_plan_s *p, int rate, UnitKind kind, DevTable **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ZFPX_ECUDA;
    const long long key = ((long long)dev << 32) | ((long long)(rate + 1024) << 4) | (long long)kind;
    std::lock_guard<std::mutex> g(p->mu);
    auto it = p->tables.find(key);
    if (it != p->tables.end()) { *out = &it->second; return ZFPX_OK; }
    std::vector<MsgDev> h;
    const int64_t units = host_table(p, rate, kind, {}, h);
    DevTable t;
    const int rc = upload_table(h, units, &t);
    if (rc) return rc;
    auto res = p->tables.emplace(key, t);
    *out = &res.first->second;
    return ZFPX_OK;
}

}  // namespace zfpx

using namespace zfpx;

extern "C" {

const char *zfpx_strerror(int code)
{
    switch (code) {
    case ZFPX_OK: return "ok";
    case ZFPX_EINVAL: return "invalid argument";
    case ZFPX_ESIZE: return "buffer too small";
    case ZFPX_ECUDA: return "CUDA error";
    case ZFPX_ETIMEOUT: return "bounded device wait expired";
    case ZFPX_ENOMEM_BUDGET: return "request exceeds the admission budget";
    case ZFPX_ENOMEM: return "out of memory";
    default: return "unknown error";
    }
}

uint64_t zfpx_launch_count(void) { return g_launches.load(); }

int zfpx_plan_create(zfpx_plan *out, const zfpx_view3 *src, const zfpx_view3 *dst,
                     int pr, int pc, int transposition, int dims, int split_mode)
{
    if (!out || !src || !dst) return ZFPX_EINVAL;
    *out = nullptr;
    if (pr < 1 || pc < 1 || (long long)pr * pc > (1 << 20)) return ZFPX_EINVAL;
    if (transposition != 0 && transposition != 1) return ZFPX_EINVAL;
    if (dims < 1 || dims > 3) return ZFPX_EINVAL;
    if (split_mode != ZFPX_SPLIT_BALANCED && split_mode != ZFPX_SPLIT_TABLE1) return ZFPX_EINVAL;
    for (int a = 0; a < 3; a++) {
        if (src->n[a] < 1 || src->n[a] != dst->n[a] || src->n[a] > kMaxExtent) return ZFPX_EINVAL;
        if (src->stride[a] < 0 || dst->stride[a] < 0) return ZFPX_EINVAL;
    }
    if ((int64_t)pr * pc * (transposition == 0 ? pc : pr) > kMaxMessages) return ZFPX_EINVAL;
    zfpx_plan_s *p = new (std::nothrow) zfpx_plan_s;
    if (!p) return ZFPX_ENOMEM;
    for (int a = 0; a < 3; a++) { p->n[a] = src->n[a]; p->ss[a] = src->stride[a]; p->ds[a] = dst->stride[a]; }
    p->pr = pr; p->pc = pc; p->P = pr * pc;
    p->transposition = transposition; p->dims = dims; p->split_mode = split_mode;

    std::vector<int64_t> xs, xl, ys, yl, zs, zl;
    try {
        if (transposition == 0) {
            split(p->n[0], pc, split_mode, xs, xl);
            split(p->n[1], pr, split_mode, ys, yl);
            split(p->n[2], pc, split_mode, zs, zl);
            // source rank j*pc+i, in send order: by source, then destination peer k
            for (int j = 0; j < pr; j++)
                for (int i = 0; i < pc; i++)
                    for (int k = 0; k < pc; k++)
                        p->msgs.push_back(HostMsg{j * pc + i, j * pc + k, i, k,
                                                  xs[i], xl[i], ys[j], yl[j], zs[k], zl[k]});
        } else {
            split(p->n[0], pr, split_mode, xs, xl);
            split(p->n[1], pr, split_mode, ys, yl);
            split(p->n[2], pc, split_mode, zs, zl);
            for (int j = 0; j < pr; j++)
                for (int k = 0; k < pc; k++)
                    for (int l = 0; l < pr; l++)
                        p->msgs.push_back(HostMsg{j * pc + k, l * pc + k, j, l,
                                                  xs[l], xl[l], ys[j], yl[j], zs[k], zl[k]});
        }
    } catch (const std::bad_alloc &) {
        delete p;
        return ZFPX_ENOMEM;
    }
    // The kernels index a message's 4-value groups along x (1-D blocks, the
    // packs' quads; every coarser block count and row count is at most this)
    // with 32-bit integers.
    for (const HostMsg &m : p->msgs) {
        const int64_t g = ceil4(m.nx) * m.ny;                     // <= 2^29 * 2^31: no overflow
        if (g > INT32_MAX || g * m.nz > INT32_MAX) {
            delete p;
            return ZFPX_EINVAL;
        }
    }
    *out = p;
    return ZFPX_OK;
}

void zfpx_plan_destroy(zfpx_plan p)
{
    if (!p) return;
    for (auto &kv : p->tables)
        if (kv.second.d_msgs) cudaFree(kv.second.d_msgs);
    delete p;
}

int zfpx_plan_prepare(zfpx_plan p, int rate)
{
    if (!p || !valid_rate(rate)) return ZFPX_EINVAL;
    DevTable *t = nullptr;
    int rc = get_table(p, rate, UNIT_CHUNK16, &t);                 // the permutation
    if (!rc) rc = get_table(p, rate, valid_codec_rate(rate) ? UNIT_BLOCKS32 : UNIT_QUADS, &t);
    return rc;
}

int zfpx_plan_num_messages(zfpx_plan p) { return p ? (int)p->msgs.size() : ZFPX_EINVAL; }

int zfpx_plan_message(zfpx_plan p, int i, int32_t ranks[4], int64_t box[6])
{
    if (!p || i < 0 || i >= (int)p->msgs.size() || !ranks || !box) return ZFPX_EINVAL;
    const HostMsg &m = p->msgs[i];
    ranks[0] = m.src; ranks[1] = m.dst; ranks[2] = m.src_peer; ranks[3] = m.dst_peer;
    box[0] = m.x0; box[1] = m.nx; box[2] = m.y0; box[3] = m.ny; box[4] = m.z0; box[5] = m.nz;
    return ZFPX_OK;
}

static int find_msg(zfpx_plan p, int src, int dst)
{
    for (size_t i = 0; i < p->msgs.size(); i++)
        if (p->msgs[i].src == src && p->msgs[i].dst == dst) return (int)i;
    return -1;
}

size_t zfpx_message_bytes(zfpx_plan p, int rate, int src, int dst)
{
    if (!p || !valid_rate(rate)) return 0;
    int i = find_msg(p, src, dst);
    return i < 0 ? 0 : (size_t)message_bytes(p, p->msgs[i], rate);
}

int64_t zfpx_message_offset(zfpx_plan p, int rate, int layout, int src, int dst)
{
    if (!p || !valid_rate(rate) || (layout != ZFPX_LAYOUT_SEND && layout != ZFPX_LAYOUT_RECV)) return -1;
    int i = find_msg(p, src, dst);
    if (i < 0) return -1;
    return layout_offsets(p, rate, layout, nullptr)[i];
}

size_t zfpx_buffer_bytes(zfpx_plan p, int rate)
{
    if (!p || !valid_rate(rate)) return 0;
    return (size_t)buffer_bytes(p, rate);
}

}  // extern "C"
