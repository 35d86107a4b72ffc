// Device-side construction of the SELL-32 copies used by the row kernels (sell_build.cu).
#pragma once
#include "core.cuh"

namespace hprqp {

// SELL-32 copy of a device CSR matrix (the layout of the row kernels' SELL schedule):
// sell_layout fills perm (slices*32 ints), width (slices), off (slices+1) and *total (the
// entry count); sell_fill then writes the entries into zeroed sci / sv of *total each
cudaError_t sell_layout(const Csr& M, int* perm, int* width, int* off, long long* total, cudaStream_t s);
cudaError_t sell_fill(const Csr& M, const int* perm, const int* off, int* sci, double* sv, cudaStream_t s);

// Tiled SELL copy (SellTiles) of a device CSR matrix over column tiles of width W (ntile <=
// kMaxTilesDevice): tile_layout fills len and slot (ntile * rows), perm (ntile * slices * 32),
// width (ntile * slices), off (ntile * (slices + 1)) and *total; tile_fill then writes the
// entries into zeroed col / val of *total each.
constexpr int kMaxTilesDevice = 64;
cudaError_t tile_layout(const Csr& M, int W, int ntile, int* len, int* perm, int* slot, int* width, int* off,
                        long long* total, cudaStream_t s);
cudaError_t tile_fill(const Csr& M, int W, int ntile, const int* slot, const int* off, unsigned short* col,
                      double* val, cudaStream_t s);

// Transpose T (cols x rows) of a device CSR matrix M, each row of T in increasing row order of
// M: transpose_layout fills rpT (cols + 1) and *maxlen (the longest row of T); transpose_fill
// then writes ciT / vT (M.nnz each), sorting each row of T by insertion (use the host
// transpose when *maxlen is large).
cudaError_t transpose_layout(const Csr& M, int* rpT, int* maxlen, cudaStream_t s);
cudaError_t transpose_fill(const Csr& M, const int* rpT, int* cur, int* ciT, double* vT, cudaStream_t s);

}  // namespace hprqp
