// Test helper: Philox4x32-10 words from PyTorch's header-only engine
// (ATen/core/PhiloxRNGEngine.h, at::philox_engine), an implementation
// independent of the oracle's.  Built by tests/test_oracle_pins.py with g++
// against the torch include directory; nothing in the library uses it.
//
// The engine's state is key = (seed lo, seed hi) and counter = (offset lo,
// offset hi, subsequence lo, subsequence hi); its first four outputs are the
// four words of one 10-round block of that (counter, key).
#include <ATen/core/PhiloxRNGEngine.h>

#include <cstdint>

extern "C" void torch_philox_blocks(const uint32_t *ctr, const uint32_t *key, uint32_t *out,
                                    int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t *c = ctr + 4 * i, *k = key + 2 * i;
        const uint64_t seed = (uint64_t)k[0] | ((uint64_t)k[1] << 32);
        const uint64_t offset = (uint64_t)c[0] | ((uint64_t)c[1] << 32);
        const uint64_t subseq = (uint64_t)c[2] | ((uint64_t)c[3] << 32);
        at::philox_engine e(seed, subseq, offset);
        for (int w = 0; w < 4; ++w) out[4 * i + w] = e(10);
    }
}
