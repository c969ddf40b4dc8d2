// Host build of the candidate-set refinement rule of the CUDA path
// (paper_2604_10601_gb300/csrc/refine.cuh, compiled here as plain C++), run
// in rounds the way the engine runs its kernel: every round starts from a
// copy of the previous bitmaps and clears the candidates that lost their
// support. Test harness only: tests/test_refine_host.py compares it with
// the oracle.
#include <cstdint>
#include <cstring>
#include <vector>

#include "refine.cuh"

extern "C" int refine_host(int64_t n, const int64_t* rowptr, const int32_t* col, int32_t k, const uint32_t* qadj,
                           uint32_t* bits, int32_t max_rounds) {
    const int64_t words = (n + 31) / 32;
    std::vector<uint32_t> cur(bits, bits + (size_t)k * words), nxt;
    int rounds = 0;
    for (int r = 0; r < max_rounds; ++r) {
        nxt = cur;
        bool changed = false;
        for (int64_t v = 0; v < n; ++v) {
            const uint32_t bit = 1u << (v & 31);
            uint32_t in = 0;
            for (int u = 0; u < k; ++u)
                if (cur[(size_t)u * words + (v >> 5)] & bit) in |= 1u << u;
            if (!in) continue;
            uint32_t drop = in & ~sgm_refine_vertex(rowptr, col, v, cur.data(), words, k, qadj, in);
            if (drop) changed = true;
            while (drop) {
                const int u = sgm_low_bit(drop);
                drop &= drop - 1u;
                nxt[(size_t)u * words + (v >> 5)] &= ~bit;
            }
        }
        if (!changed) break;
        ++rounds;
        cur.swap(nxt);
    }
    std::memcpy(bits, cur.data(), sizeof(uint32_t) * cur.size());
    return rounds;
}
