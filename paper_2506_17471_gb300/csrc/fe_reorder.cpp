// Host-side mesh orderings for gather locality.
//
// At low order the action is dominated by the indirect gathers and scatters of
// Algorithm 2: each DoF is read and updated once per cell that contains it, and
// how often those accesses hit the caches depends on how close in memory the
// DoFs of cells processed together are (Sec. "Behavior at low orders" suggests
// an order of cells and DoFs that keeps cells sharing DoFs close).  Two
// orderings are provided:
//   * cells along a Morton (Z-order) curve of their centroids, so that the 32
//     cells of a warp and the cells of neighbouring warps are spatial
//     neighbours;
//   * entities (nodes or vertices) numbered by first touch in a given cell
//     order, so that the entities of consecutive cells get consecutive indices.
// Both are permutations; applying them changes the memory layout only (the
// action is the same operator up to the renumbering).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "fe_internal.h"

namespace {

// Spreads the low 21 bits of v so that bit i lands at bit 3i (3D) or the low 32
// bits at 2i (2D).
uint64_t spread3(uint64_t v)
{
    v &= 0x1FFFFFull;
    v = (v | (v << 32)) & 0x1F00000000FFFFull;
    v = (v | (v << 16)) & 0x1F0000FF0000FFull;
    v = (v | (v << 8)) & 0x100F00F00F00F00Full;
    v = (v | (v << 4)) & 0x10C30C30C30C30C3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

uint64_t spread2(uint64_t v)
{
    v &= 0xFFFFFFFFull;
    v = (v | (v << 16)) & 0x0000FFFF0000FFFFull;
    v = (v | (v << 8)) & 0x00FF00FF00FF00FFull;
    v = (v | (v << 4)) & 0x0F0F0F0F0F0F0F0Full;
    v = (v | (v << 2)) & 0x3333333333333333ull;
    v = (v | (v << 1)) & 0x5555555555555555ull;
    return v;
}

}  // namespace

extern "C" int fe_order_cells_morton(int dim, int n_vertices, int n_cells, const double *coords,
                                     const int32_t *cell2vertex, int32_t *perm)
{
    if ((dim != 2 && dim != 3) || n_vertices < 0 || n_cells < 0) return FE_ERR_INVALID_ARG;
    if (n_cells > 0 && (!coords || !cell2vertex || !perm)) return FE_ERR_INVALID_ARG;
    const int nv = dim + 1;
    // centroids and their bounding box
    std::vector<double> cen((size_t)n_cells * dim);
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int c = 0; c < n_cells; ++c) {
        for (int i = 0; i < dim; ++i) {
            double s = 0.0;
            for (int m = 0; m < nv; ++m) {
                const int v = cell2vertex[(size_t)c * nv + m];
                if (v < 0 || v >= n_vertices) return FE_ERR_INDEX;
                s += coords[(size_t)v * dim + i];
            }
            s /= nv;
            if (!std::isfinite(s)) return FE_ERR_BAD_MESH;
            cen[(size_t)c * dim + i] = s;
            lo[i] = std::min(lo[i], s);
            hi[i] = std::max(hi[i], s);
        }
    }
    // quantise each coordinate to 21 (3D) or 32 (2D) bits and interleave
    const double levels = dim == 3 ? 2097151.0 : 4294967295.0;
    std::vector<std::pair<uint64_t, int32_t>> key((size_t)n_cells);
    for (int c = 0; c < n_cells; ++c) {
        uint64_t k = 0;
        for (int i = 0; i < dim; ++i) {
            const double ext = hi[i] - lo[i];
            const double t = ext > 0.0 ? (cen[(size_t)c * dim + i] - lo[i]) / ext : 0.0;
            const uint64_t q = (uint64_t)std::llround(std::min(std::max(t, 0.0), 1.0) * levels);
            k |= (dim == 3 ? spread3(q) : spread2(q)) << i;
        }
        key[(size_t)c] = {k, c};
    }
    // ties keep the original order (pairs compare by key, then index)
    std::sort(key.begin(), key.end());
    for (int k = 0; k < n_cells; ++k) perm[k] = key[(size_t)k].second;
    return FE_OK;
}

extern "C" int fe_order_first_touch(int n_entities, int n_cells, int per_cell, const int32_t *cell2entity,
                                    const int32_t *cell_order, int32_t *new_of_old)
{
    if (n_entities < 0 || n_cells < 0 || per_cell < 1) return FE_ERR_INVALID_ARG;
    if ((n_cells > 0 && !cell2entity) || (n_entities > 0 && !new_of_old)) return FE_ERR_INVALID_ARG;
    std::vector<char> seen_cell(cell_order ? (size_t)n_cells : 0, 0);
    for (int e = 0; e < n_entities; ++e) new_of_old[e] = -1;
    int32_t next = 0;
    for (int k = 0; k < n_cells; ++k) {
        const int c = cell_order ? cell_order[k] : k;
        if (c < 0 || c >= n_cells) return FE_ERR_INDEX;
        if (cell_order) {
            if (seen_cell[(size_t)c]) return FE_ERR_INVALID_ARG;   // not a permutation
            seen_cell[(size_t)c] = 1;
        }
        for (int j = 0; j < per_cell; ++j) {
            const int e = cell2entity[(size_t)c * per_cell + j];
            if (e < 0 || e >= n_entities) return FE_ERR_INDEX;
            if (new_of_old[e] < 0) new_of_old[e] = next++;
        }
    }
    // entities no cell references keep their relative order after the others
    for (int e = 0; e < n_entities; ++e)
        if (new_of_old[e] < 0) new_of_old[e] = next++;
    return FE_OK;
}
