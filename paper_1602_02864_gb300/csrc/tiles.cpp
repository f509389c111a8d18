// tiles.cpp -- import of the paper's tiled SCSR + COO storage (Section 3.2).
//
// Section 3.2 stores the matrix in t x t tiles (t <= 32768).  Inside a tile,
// every non-empty row with two or more entries is a row header (a 16-bit word
// with the most significant bit set, the low 15 bits the row within the
// tile) followed by its column words (most significant bit clear); rows with
// a single entry are stored afterwards in coordinate form, as (row, column)
// word pairs, so reading them needs no end-of-row test.  Values, if any, follow
// the same order.  The importer decodes every tile into the library's CSR
// (entries of a row keep tile order, then storage order) and creates a
// resident handle; the tile layout itself is not used on the GPU.
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace spmm {
int create_from_host_csr(spmm_mat** out, int64_t n_rows, int64_t n_cols, int64_t nnz, const int64_t* row_ptr,
                         const int32_t* col_idx, const void* values, spmm_dtype vtype, uint32_t flags,
                         const spmm_opts* opts, cudaStream_t s, const char* who);
}

using namespace spmm;

extern "C" int spmm_create_tiles(spmm_mat_t* out, int64_t n_rows, int64_t n_cols, int32_t tile, int64_t n_tiles,
                                 const spmm_tile_desc* tiles, spmm_dtype vtype, uint32_t flags,
                                 const spmm_opts* opts, void* stream) {
    set_error("");
    if (!out || (n_tiles > 0 && !tiles) || n_tiles < 0 || n_rows < 0 || n_cols < 1) {
        set_error("spmm_create_tiles: NULL argument or bad size");
        return SPMM_ERR_ARG;
    }
    if (tile < 1 || tile > 32768) {
        set_error("spmm_create_tiles: tile size must be 1..32768 (15-bit row and column words)");
        return SPMM_ERR_ARG;
    }
    const bool has_val = n_tiles > 0 && tiles[0].values != nullptr;
    size_t vsize = 0;
    if (has_val) {
        if (vtype == SPMM_F32) vsize = 4;
        else if (vtype == SPMM_BF16 || vtype == SPMM_F16) vsize = 2;
        else { set_error("spmm_create_tiles: values must be F32, BF16 or F16"); return SPMM_ERR_ARG; }
    }
    // ---- pass 1: validate and count entries per row
    std::vector<int64_t> cnt((size_t)n_rows + 1, 0);
    int64_t nnz = 0;
    auto bad = [&](int64_t t, const char* why) {
        set_error("spmm_create_tiles: tile " + std::to_string(t) + ": " + why);
        return SPMM_ERR_FORMAT;
    };
    for (int64_t t = 0; t < n_tiles; ++t) {
        const spmm_tile_desc& d = tiles[t];
        if ((d.values != nullptr) != has_val) return bad(t, "values given for some tiles only");
        if (d.n_scsr_words < 0 || d.n_coo < 0 || (d.n_scsr_words + d.n_coo > 0 && !d.data))
            return bad(t, "negative section size or NULL data");
        const int64_t rbase = d.tile_row * tile, cbase = d.tile_col * tile;
        if (d.tile_row < 0 || d.tile_col < 0 || rbase >= std::max<int64_t>(n_rows, 1) || cbase >= n_cols)
            return bad(t, "tile position outside the matrix");
        int64_t row = -1, row_len = 0;
        for (int64_t w = 0; w < d.n_scsr_words; ++w) {
            const uint16_t v = d.data[w];
            if (v & 0x8000u) {
                if (row >= 0 && row_len == 0) return bad(t, "row header without columns");
                row = v & 0x7fff;
                row_len = 0;
                if (row >= tile || rbase + row >= n_rows) return bad(t, "row outside the tile or matrix");
            } else {
                if (row < 0) return bad(t, "column word before the first row header");
                if ((int64_t)v >= tile || cbase + v >= n_cols) return bad(t, "column outside the tile or matrix");
                ++cnt[(size_t)(rbase + row)];
                ++row_len;
                ++nnz;
            }
        }
        if (row >= 0 && row_len == 0) return bad(t, "row header without columns");
        for (int64_t j = 0; j < d.n_coo; ++j) {
            const uint16_t r = d.data[d.n_scsr_words + 2 * j], c = d.data[d.n_scsr_words + 2 * j + 1];
            if ((r & 0x8000u) || (c & 0x8000u)) return bad(t, "coordinate words must have the top bit clear");
            if (r >= tile || c >= tile || rbase + r >= n_rows || cbase + c >= n_cols)
                return bad(t, "coordinate entry outside the tile or matrix");
            ++cnt[(size_t)(rbase + r)];
            ++nnz;
        }
    }
    // ---- pass 2: fill CSR in tile order, storage order within a tile
    std::vector<int64_t> rp((size_t)n_rows + 1, 0);
    for (int64_t i = 0; i < n_rows; ++i) rp[(size_t)i + 1] = rp[(size_t)i] + cnt[(size_t)i];
    std::vector<int64_t> pos(rp.begin(), rp.end() - 1);
    std::vector<int32_t> ci((size_t)nnz);
    std::vector<char> va(has_val ? (size_t)nnz * vsize : 0);
    for (int64_t t = 0; t < n_tiles; ++t) {
        const spmm_tile_desc& d = tiles[t];
        const int64_t rbase = d.tile_row * tile, cbase = d.tile_col * tile;
        const char* vals = static_cast<const char*>(d.values);
        int64_t k = 0, row = 0;
        auto put = [&](int64_t r, int64_t c) {
            const int64_t q = pos[(size_t)r]++;
            ci[(size_t)q] = (int32_t)c;
            if (has_val) std::memcpy(&va[(size_t)q * vsize], vals + k * vsize, vsize);
            ++k;
        };
        for (int64_t w = 0; w < d.n_scsr_words; ++w) {
            const uint16_t v = d.data[w];
            if (v & 0x8000u) row = v & 0x7fff;
            else put(rbase + row, cbase + v);
        }
        for (int64_t j = 0; j < d.n_coo; ++j)
            put(rbase + d.data[d.n_scsr_words + 2 * j], cbase + d.data[d.n_scsr_words + 2 * j + 1]);
    }
    return create_from_host_csr(out, n_rows, n_cols, nnz, rp.data(), ci.data(), has_val ? va.data() : nullptr,
                                vtype, flags, opts, (cudaStream_t)stream, "spmm_create_tiles");
}
