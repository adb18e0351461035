// Host check of the multiply-high division the plan kernels use for block
// indices (block_divisor in paper_2609_24294_gb300/csrc/zfpx_internal.h sets
// the constants; the kernels' divu computes t = mulhi(n, m), then
// (t + ((n - t) >> 1)) >> (l - 1), or n itself when l = 0), driven by
// tests/test_divisor_host.py.  Test infrastructure only.
//
//   divisor_host < pairs > quotients   (pairs: uint32 d, uint32 n; quotients: uint32)
// Exit status 0, or 2 on bad input.
#include <cstdint>
#include <cstdio>
#include <vector>

#include "zfpx_internal.h"

int main()
{
    std::vector<uint32_t> in;
    uint32_t buf[2];
    while (fread(buf, sizeof(uint32_t), 2, stdin) == 2) in.insert(in.end(), buf, buf + 2);
    for (size_t i = 0; i < in.size(); i += 2) {
        const uint32_t d = in[i], n = in[i + 1];
        if (d == 0) return 2;
        uint32_t m;
        int32_t l;
        zfpx::block_divisor(d, m, l);
        const uint32_t t = (uint32_t)(((uint64_t)n * m) >> 32);
        const uint32_t q = l ? (t + ((n - t) >> 1)) >> (l - 1) : n;
        fwrite(&q, sizeof q, 1, stdout);
    }
    return 0;
}
