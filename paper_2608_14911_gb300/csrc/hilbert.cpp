// Hilbert-curve ranks of the cells of a box, used as the storage order of the
// particles (paper "Performance optimizations": data sorting for locality).
//
// The curve index of a cell follows J. Skilling, "Programming the Hilbert
// curve", AIP Conf. Proc. 707, 381 (2004): the coordinates are transformed in
// place to the "transposed" Hilbert index (undo the excess work of each level,
// then Gray-encode), and the index is read off by interleaving their bits.
// Grids that are not powers of two use the curve of the enclosing 2^b cube and
// keep the relative order of the cells that exist.
#include <algorithm>
#include <cstdint>
#include <numeric>
#include <vector>

#include "../../include/espp.h"

namespace espp {

static uint64_t hilbert_index3(uint32_t x, uint32_t y, uint32_t z, int bits) {
    uint32_t X[3] = {x, y, z};
    const uint32_t M = 1u << (bits - 1);
    // undo excess work, from the top level down
    for (uint32_t Q = M; Q > 1; Q >>= 1) {
        const uint32_t P = Q - 1;
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;  // invert the low bits of the first axis
            } else {
                const uint32_t t = (X[0] ^ X[i]) & P;  // exchange low bits
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    // Gray encode
    for (int i = 1; i < 3; ++i) X[i] ^= X[i - 1];
    uint32_t t = 0;
    for (uint32_t Q = M; Q > 1; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1;
    for (int i = 0; i < 3; ++i) X[i] ^= t;
    // interleave: the most significant bit of axis 0 comes first
    uint64_t h = 0;
    for (int b = bits - 1; b >= 0; --b)
        for (int i = 0; i < 3; ++i) h = (h << 1) | ((X[i] >> b) & 1u);
    return h;
}

void hilbert_ranks(int nx, int ny, int nz, int* rank) {
    int m = std::max(nx, std::max(ny, nz));
    int bits = 1;
    while ((1 << bits) < m) ++bits;
    const int64_t n = (int64_t)nx * ny * nz;
    std::vector<uint64_t> key((size_t)n);
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                key[((size_t)z * ny + y) * nx + x] = hilbert_index3(x, y, z, bits);
    std::vector<int64_t> order((size_t)n);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return key[a] < key[b]; });
    for (int64_t r = 0; r < n; ++r) rank[order[r]] = (int)r;
}

}  // namespace espp

extern "C" int espp_hilbert_ranks(int32_t nx, int32_t ny, int32_t nz, int32_t* rank) {
    if (nx <= 0 || ny <= 0 || nz <= 0 || !rank) return ESPP_ERR_ARG;
    espp::hilbert_ranks(nx, ny, nz, rank);
    return ESPP_OK;
}
