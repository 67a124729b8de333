// Generation of bitsliced XOR schedules (host side).
//
// Multiplication by a constant c is the 8x8 bit matrix M_c whose column j
// holds the bits of c * 2^j; with an input byte column cut into eight bit
// planes p0..p7, output plane i of c*x is the XOR of the planes j with
// M_c[i][j] = 1.  Splitting j into 0..3 and 4..7, every such XOR is
// Q[a] ^ R[b] where Q (R) holds the XORs of all subsets of p0..p3 (p4..p7)
// and a, b are the two nibbles of row i of M_c.  For each dense block of a
// matrix (at most 8 rows sharing their inputs) the emitter writes a device
// function that walks the block's inputs and accumulates those terms, and a
// persistent kernel over the blocks (bitslice_dev.cuh supplies the rest).
//
// Used at build time for the built-in encode matrices (gen_bitslice.cpp) and
// at run time for matrices known only then (jit.cpp).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace pmrc {

constexpr int kBsEmitRows = 8;        // rows per block (8 x 8 bit-plane accumulators)
constexpr int kBsEmitMaxBlocks = 64;  // bitslice_dev.cuh: kBsMaxBlocks

struct BsBlock {
  std::vector<int> rows, inputs;
};

// Rows with the same non-zero columns form a group; each group is cut into
// blocks of at most 8 rows (encode matrices: the rows of one slot share the
// symbols of one column of the message matrix).
std::vector<BsBlock> bs_blocks_by_support(const uint8_t *M, int rows, int cols);

// Consecutive rows in blocks of at most 8, each reading the union of its
// rows' non-zero columns (dense matrices such as reconstruction rows).
std::vector<BsBlock> bs_blocks_chunked(const uint8_t *M, int rows, int cols);

// Rows grouped by their non-zero columns other than own[r] (a column of
// each row's own, such as the received parity block a row starts from), in
// order of first appearance; groups packed whole into blocks of at most 8
// rows whose inputs stay within max_inputs (a block holding one group may
// exceed it), a group of more than 8 cut into balanced blocks of its own;
// each block reads the union of its rows' columns.
std::vector<BsBlock> bs_blocks_grouped(const uint8_t *M, int rows, int cols,
                                       const std::vector<int> &own, int max_inputs);

// The launch's work items g = b * ntiles + t (block b < nblocks, 1 KiB
// column tile t < ntiles) cut into ncta contiguous ranges of about equal
// cost (cost[b] per tile of block b): CTA c takes [cta_g[c], cta_g[c+1]),
// with cta_g[0] = 0 <= cta_g[1] <= ... <= cta_g[ncta] = nblocks * ntiles.
// Host only (the launcher's schedule; tested on the CPU).
void bs_cta_ranges(int nblocks, const int *cost, uint64_t ntiles, int ncta, uint32_t *cta_g);

struct BsEmitted {
  std::string code;       // block functions and the kernel
  std::vector<int> cost;  // relative cost of each block per warp tile
  long long xors = 0;     // XOR operations per 32-byte column
};

// Source of the block functions and of the kernel `name` for the matrix M
// (rows x cols, row-major): output row r goes to pointer slot cols + r.  With
// extern_c the kernel gets C linkage (for lookup by name after run-time
// compilation).  With pair_split the two warps of a pair take each (block,
// tile) item together, each over half of the block's inputs, and combine
// their partial sums through shared memory (kBsPairExchangeBytes beyond the
// staging ring): twice the warp tasks at half the latency, for launches
// with few tiles per warp.  in_planes / out_planes: the inputs are, the
// outputs are stored as, plane-layout blocks (each lane's 32 bytes hold the
// eight 32-bit bit planes of those 32 byte columns) -- the intermediate of
// a two-launch product, which skips the transposes on both sides of it.
BsEmitted bs_emit_kernel(const uint8_t *M, int rows, int cols, const std::vector<BsBlock> &blks,
                         const std::string &name, bool extern_c, bool pair_split = false,
                         bool in_planes = false, bool out_planes = false);
constexpr int kBsPairExchangeBytes = 8 * 8 * 8 * 32 * 4;  // 8 pairs x 8 rows x 8 planes x 32 lanes

// Repair schedules, emitted at run time for one failed node's helper
// coefficients phi (alpha entries, the projection each helper applies to its
// alpha blocks, Sec. 2/3.3) and, for the fused kernel, the newcomer matrix D
// (alpha x d, row-major).  Each helper block that phi reads is turned into
// bit planes once and multiplied by its constant phi[j] as plain XORs of
// planes (output plane i of c*x is the XOR of the input planes jj with bit i
// of c*2^jj set); no subset tables are needed for a single row.
//
// Projection kernel: warp task = (1 KiB column tile, group of
// kBsHelpersPerTask helpers); helper h's blocks at pointer slots
// [h*alpha, h*alpha + alpha), its projection to slot nh*alpha + h.
//
// Fused repair kernel (alpha <= 8): the two warps of a pair take the same
// tile, each the projections of half the helpers, which stay in registers
// and go straight into the newcomer's apply (subset tables of the
// projection, one 3-input XOR per output plane); the two partial sums are
// combined through shared memory.  Output row r goes to slot d*alpha + r.
constexpr int kBsHelpersPerTask = 2;
constexpr int kBsFusedMaxAlpha = 8;

BsEmitted bs_emit_projection(const uint8_t *phi, int alpha, const std::string &name);
BsEmitted bs_emit_fused_repair(const uint8_t *phi, int alpha, const uint8_t *D, int d,
                               const std::string &name);

}  // namespace pmrc
