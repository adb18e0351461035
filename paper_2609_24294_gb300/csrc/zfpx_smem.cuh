// Per-lane shared-memory views used by the codec kernels (codec.cu, batch.cu).
// Every warp owns its tiles; lane l works in its own column, so no view
// needs a barrier other than the warp's own __syncwarp around the copies in
// and out of a tile.
#pragma once
#include <cstdint>

namespace zfpx {

// Writer into this lane's column of a [word][lane] tile of RATE + 2 64-bit
// words (RATE stream words, two slack words past the budget), XOR-swizzled (word w of lane l at w * 32 + (l ^ w)) so that both the
// per-lane writes and the warp's coalesced copy-out spread over the banks.
// put(bits, len): 1 <= len <= 64, bits < 2^len; zeros(len): len >= 0;
// finish(): flush and zero-fill to RATE words; orw(i, v): OR v into word i
// (only after finish()).
template <int RATE>
struct SmemWriter {
    uint64_t *sm;
    uint64_t acc;
    int nb, w, lane;
    __device__ __forceinline__ uint64_t &word(int i) const { return sm[i * 32 + (lane ^ i)]; }
    __device__ __forceinline__ void put(uint64_t bits, int len)
    {
        acc |= bits << nb;
        int t = nb + len;
        if (t >= 64) {
            word(w) = acc;
            w++;
            acc = nb ? (bits >> (64 - nb)) : 0ull;
            t -= 64;
        }
        nb = t;
    }
    __device__ __forceinline__ void zeros(int len)
    {
        int t = nb + len;
        while (t >= 64) {
            word(w) = acc;
            w++;
            acc = 0ull;
            t -= 64;
        }
        nb = t;
    }
    __device__ __forceinline__ void finish()
    {
        if (nb > 0) { word(w) = acc; w++; }
        for (; w < RATE; w++) word(w) = 0ull;
    }
    __device__ __forceinline__ void orw(int i, uint64_t v) const { word(i) |= v; }
};

// Bit planes of one block in this lane's column of a [plane][lane] tile
// (a warp touches 32 consecutive words: conflict-free).
struct SmemPlanes {
    uint64_t *sm;
    int lane;
    __device__ __forceinline__ void store(int k, uint64_t X) { sm[k * 32 + lane] = X; }
    __device__ __forceinline__ uint64_t load(int k) const { return sm[k * 32 + lane]; }
    // the low (half 0) or high (half 1) 32 bits of plane k
    __device__ __forceinline__ void store_half(int k, int half, uint32_t v)
    {
        reinterpret_cast<uint32_t *>(sm)[2 * (k * 32 + lane) + half] = v;
    }
    __device__ __forceinline__ uint32_t load_half(int k, int half) const
    {
        return reinterpret_cast<const uint32_t *>(sm)[2 * (k * 32 + lane) + half];
    }
};

// 32-bit bit planes (2-D blocks: 16 coefficients) in this lane's column of a
// [plane][lane] tile; the same interface as the low half of SmemPlanes.
struct SmemPlanes16 {
    uint32_t *sm;
    int lane;
    __device__ __forceinline__ void store_half(int k, int, uint32_t v) { sm[k * 32 + lane] = v; }
    __device__ __forceinline__ uint32_t load_half(int k, int) const { return sm[k * 32 + lane]; }
};

// Stream tile of one warp: 32-bit words in a [word][lane] layout (word i of
// lane l at i * 32 + l), so every lane reads its own column without bank
// conflicts; two zero rows follow the stream, so the 64-bit window read at
// any position before the stream's end stays inside the tile.
struct StreamTile {
    const uint32_t *sm;
    int lane;
    __device__ __forceinline__ uint32_t get(int i) const { return sm[i * 32 + lane]; }
};

}  // namespace zfpx
