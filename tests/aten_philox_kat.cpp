// Known-answer source for the oracle's Philox4x32-10: PyTorch's open-source
// (BSD) philox_engine from ATen/core/PhiloxRNGEngine.h, an implementation
// written independently of this project. Reads lines "c0 c1 c2 c3 k0 k1"
// and prints the four 32-bit output words of the block with that counter
// and key. The engine's (seed, subsequence, offset) map onto the block as
// key = (seed lo, seed hi), counter = (offset lo, offset hi, subsequence lo,
// subsequence hi); its first four calls return the block's words in order.
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdint>
#include <cstdio>

int main()
{
    unsigned long c0, c1, c2, c3, k0, k1;
    while (std::scanf("%lu %lu %lu %lu %lu %lu", &c0, &c1, &c2, &c3, &k0, &k1) == 6) {
        const uint64_t seed = (uint64_t)k0 | ((uint64_t)k1 << 32);
        const uint64_t subsequence = (uint64_t)c2 | ((uint64_t)c3 << 32);
        const uint64_t offset = (uint64_t)c0 | ((uint64_t)c1 << 32);
        at::philox_engine e(seed, subsequence, offset);
        const uint32_t w0 = e(), w1 = e(), w2 = e(), w3 = e();
        std::printf("%u %u %u %u\n", w0, w1, w2, w3);
    }
    return 0;
}
