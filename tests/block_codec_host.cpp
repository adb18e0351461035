// Host build of the library's block coders: the __host__ __device__ functions
// of paper_2609_24294_gb300/csrc/zfpx_block.cuh compiled by a C++ compiler for
// the CPU, driven by tests/test_block_codec_host.py, which compares what they
// produce with the oracle.  Test infrastructure only.
//
//   block_codec_host MODE RATE < input > output      (RATE 8 or 16)
//     enc3: N x 64 float32             -> N streams of 8 RATE bytes (the scalar two-pass 3-D
//                                         encoder, the statement the GPU's warp-uniform coder follows)
//     dec3: N streams of 8 RATE bytes  -> N x 64 float32 (the GPU decoders' 3-D block decoder)
//     enc2: N x 16 float32             -> N streams of 2 RATE bytes
//     dec2: N streams of 2 RATE bytes  -> N x 16 float32
//     enc1: N x 4 float32              -> N streams of RATE / 2 bytes (four blocks in lockstep,
//                                         checked against one block at a time)
//     dec1: N streams of RATE / 2 bytes -> N x 4 float32 (likewise)
// Values in a block are in the order i + 4 j + 16 k (i fastest); streams are
// the blocks' bits LSB first in little-endian bytes.  Exit status 0 on
// success, 2 on bad arguments or input, 3 when the lockstep and one-block 1-D
// coders disagree.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "zfpx_block.cuh"

using namespace zfpx::blk;

namespace {

// A stream tile: 32-bit words, zero past the stream.
struct Tile {
    const uint32_t *w;
    uint32_t get(int i) const { return w[i]; }
};

// 64 bit planes, also addressed as 32-bit halves (half 0 = low bits).
struct Planes64 {
    uint64_t s[64];
    void store(int k, uint64_t x) { s[k] = x; }
    uint64_t load(int k) const { return s[k]; }
    void store_half(int k, int h, uint32_t v)
    {
        s[k] = h ? ((s[k] & 0xffffffffull) | ((uint64_t)v << 32)) : ((s[k] & ~0xffffffffull) | v);
    }
    uint32_t load_half(int k, int h) const { return (uint32_t)(s[k] >> (32 * h)); }
};

// 32 planes of 32 bits (2-D blocks); the half argument is not used.
struct Planes32 {
    uint32_t s[32];
    void store_half(int k, int, uint32_t v) { s[k] = v; }
    uint32_t load_half(int k, int) const { return s[k]; }
};

// The coders' bit writer: put(bits, len), zeros(len), finish() (flush and
// zero-fill to NW words), orw(i, v) (OR into word i after finish); slack words
// past NW catch a last plane that runs past the budget.
template <int NW>
struct Writer {
    uint64_t wd[NW + 4];
    uint64_t acc;
    int nb, w;
    void put(uint64_t bits, int len)
    {
        acc |= bits << nb;
        int t = nb + len;
        if (t >= 64) {
            wd[w++] = acc;
            acc = nb ? (bits >> (64 - nb)) : 0ull;
            t -= 64;
        }
        nb = t;
    }
    void zeros(int len)
    {
        int t = nb + len;
        while (t >= 64) {
            wd[w++] = acc;
            acc = 0ull;
            t -= 64;
        }
        nb = t;
    }
    void finish()
    {
        if (nb > 0) wd[w++] = acc;
        for (; w < NW; w++) wd[w] = 0ull;
    }
    void orw(int i, uint64_t v) { wd[i] |= v; }
};

std::vector<uint8_t> read_all()
{
    std::vector<uint8_t> d;
    uint8_t buf[1 << 16];
    size_t n;
    while ((n = fread(buf, 1, sizeof buf, stdin)) > 0) d.insert(d.end(), buf, buf + n);
    return d;
}

void write_all(const void *p, size_t n) { fwrite(p, 1, n, stdout); }

void load_words(const uint8_t *src, int nbytes, uint32_t *w)
{
    for (int i = 0; i < nbytes / 4; i++)
        w[i] = (uint32_t)src[4 * i] | ((uint32_t)src[4 * i + 1] << 8) | ((uint32_t)src[4 * i + 2] << 16) |
               ((uint32_t)src[4 * i + 3] << 24);
}

void store_le(uint64_t v, int nbytes, uint8_t *dst)
{
    for (int i = 0; i < nbytes; i++) dst[i] = (uint8_t)(v >> (8 * i));
}

template <int RATE>
int enc3(const std::vector<uint8_t> &in)
{
    if (in.size() % 256) return 2;
    for (size_t o = 0; o < in.size(); o += 256) {
        float x[64];
        std::memcpy(x, &in[o], sizeof x);
        Writer<RATE> wr{};
        Planes64 pl{};
        encode_block3<RATE>(x, wr, pl);
        uint8_t out[8 * RATE];
        for (int i = 0; i < RATE; i++) store_le(wr.wd[i], 8, out + 8 * i);
        write_all(out, sizeof out);
    }
    return 0;
}

template <int RATE>
int dec3(const std::vector<uint8_t> &in)
{
    constexpr int B = 8 * RATE;
    if (in.size() % B) return 2;
    for (size_t o = 0; o < in.size(); o += B) {
        uint32_t w[2 * RATE + 4] = {};
        load_words(&in[o], B, w);
        Planes64 pl{};
        float x[64];
        decode_block3_tile<RATE>(Tile{w}, x, pl);
        write_all(x, sizeof x);
    }
    return 0;
}

template <int RATE>
int enc2(const std::vector<uint8_t> &in)
{
    constexpr int NW = RATE / 4;                         // 16 RATE bits in 64-bit words
    if (in.size() % 64) return 2;
    for (size_t o = 0; o < in.size(); o += 64) {
        float x[16];
        std::memcpy(x, &in[o], sizeof x);
        Writer<NW> wr{};
        Planes32 pl{};
        encode_block2<RATE>(x, wr, pl);
        uint8_t out[8 * NW];
        for (int i = 0; i < NW; i++) store_le(wr.wd[i], 8, out + 8 * i);
        write_all(out, sizeof out);
    }
    return 0;
}

template <int RATE>
int dec2(const std::vector<uint8_t> &in)
{
    constexpr int B = 2 * RATE;
    if (in.size() % B) return 2;
    for (size_t o = 0; o < in.size(); o += B) {
        uint32_t w[RATE / 2 + 4] = {};
        load_words(&in[o], B, w);
        Planes32 pl{};
        float x[16];
        decode_block2_tile<RATE>(Tile{w}, x, pl);
        write_all(x, sizeof x);
    }
    return 0;
}

template <int RATE>
int enc1(const std::vector<uint8_t> &in)
{
    constexpr int B = RATE / 2;
    if (in.size() % 16) return 2;
    static Plane4Enc tab;
    plane4_fill(tab, 0, 1);
    const size_t n = in.size() / 16;
    for (size_t b0 = 0; b0 < n; b0 += 4) {
        float x[4][4] = {};
        for (size_t k = 0; k < 4 && b0 + k < n; k++) std::memcpy(x[k], &in[16 * (b0 + k)], 16);
        uint64_t w[4];
        encode_blocks1<RATE, 4>(x, tab, w);
        for (size_t k = 0; k < 4 && b0 + k < n; k++) {
            float one[1][4];
            std::memcpy(one[0], x[k], 16);
            uint64_t w1[1];
            encode_blocks1<RATE, 1>(one, tab, w1);
            if (w1[0] != w[k]) return 3;
            uint8_t out[B];
            store_le(w[k], B, out);
            write_all(out, B);
        }
    }
    return 0;
}

template <int RATE>
int dec1(const std::vector<uint8_t> &in)
{
    constexpr int B = RATE / 2;
    if (in.size() % B) return 2;
    static Plane4Dec tab;
    plane4_fill(tab, 0, 1);
    const size_t n = in.size() / B;
    for (size_t b0 = 0; b0 < n; b0 += 4) {
        uint64_t w[4] = {};
        for (size_t k = 0; k < 4 && b0 + k < n; k++)
            for (int i = 0; i < B; i++) w[k] |= (uint64_t)in[B * (b0 + k) + i] << (8 * i);
        float x[4][4];
        decode_blocks1<RATE, 4>(w, tab, x);
        for (size_t k = 0; k < 4 && b0 + k < n; k++) {
            const uint64_t w1[1] = {w[k]};
            float one[1][4];
            decode_blocks1<RATE, 1>(w1, tab, one);
            if (std::memcmp(one[0], x[k], 16)) return 3;
            write_all(x[k], 16);
        }
    }
    return 0;
}

template <int RATE>
int run(const char *mode, const std::vector<uint8_t> &in)
{
    if (!std::strcmp(mode, "enc3")) return enc3<RATE>(in);
    if (!std::strcmp(mode, "dec3")) return dec3<RATE>(in);
    if (!std::strcmp(mode, "enc2")) return enc2<RATE>(in);
    if (!std::strcmp(mode, "dec2")) return dec2<RATE>(in);
    if (!std::strcmp(mode, "enc1")) return enc1<RATE>(in);
    if (!std::strcmp(mode, "dec1")) return dec1<RATE>(in);
    return 2;
}

}  // namespace

int main(int argc, char **argv)
{
    if (argc != 3) return 2;
    const std::vector<uint8_t> in = read_all();
    int rc = 2;
    if (!std::strcmp(argv[2], "8")) rc = run<8>(argv[1], in);
    else if (!std::strcmp(argv[2], "16")) rc = run<16>(argv[1], in);
    fflush(stdout);
    return rc;
}
