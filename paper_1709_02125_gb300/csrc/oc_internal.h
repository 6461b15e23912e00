// Internal data structures of liboc: datasets, queued loops, and tile plans.
// Host-only header shared by the analysis (analysis.cpp) and the executor
// (runtime.cu). Kernels see only the launch descriptors of launch.h.
#pragma once

#include <array>
#include <cstdint>
#include <string>
#include <vector>

namespace oc {

constexpr int kMaxArgs = 40;
constexpr int kMaxSamples = 64;

// A dataset (arXiv 1709.02125, Sec. 3) with the library-owned host store.
// Host and device rows share one padded layout: a slow-axis "row" (a y-line in 2-D,
// a z-plane in 3-D) holds `row_elems` elements; an x-line holds `pitch` elements
// and x = 0 sits at element `ox` of its line, on a 16-byte boundary.
struct Dat {
    int ndim = 2;
    int size[3] = {1, 1, 1};
    int hlo[3] = {0, 0, 0};
    int hhi[3] = {0, 0, 0};
    int dtype = 0;           // 0 = f64, 1 = f32
    int esz = 8;
    int periodic = 0;        // bit a: axis a periodic
    int ox = 0;              // x origin within an x-line (elements)
    long long pitch = 0;     // elements per x-line
    long long ylines = 1;    // x-lines per slow row (3-D: full y extent; 2-D: 1)
    long long row_elems = 0; // elements per slow row
    int nrows = 0;           // slow rows including halos
    int y0 = 0;              // slow index of the first row (= -hlo[slow])
    void* host = nullptr;    // pinned host store, nrows * row_elems * esz bytes
    char* host_dev = nullptr;  // the store's device mapping (null: not mapped)
    bool host_pinned = false;
    bool managed = false;    // store in managed memory (OC_FLAG_MANAGED), addressed in place
    // residency (in-core mode keeps the whole dataset in the arena)
    bool resident = false;
    long long res_off = -1;
    bool dev_valid = false;   // device copy current
    bool host_valid = true;   // host copy current
    // written first by a streamed chain under the cyclic flag: its rows were not
    // downloaded, so the host store no longer holds its values (Sec. 4.1)
    bool cyc_stale = false;
    int slow() const { return ndim - 1; }
    long long row_bytes() const { return row_elems * esz; }
    long long bytes() const { return (long long)nrows * row_bytes(); }
    int ext(int a) const { return size[a] + hlo[a] + hhi[a]; }
};

struct Arg {
    int dat = -1;             // dataset or reduction handle
    int access = 0;           // OC_READ / OC_WRITE / OC_RW / OC_REDUCE
    std::vector<std::array<int, 3>> off;
    int rmin[3] = {0, 0, 0};  // min / max offset per axis
    int rmax[3] = {0, 0, 0};
};

struct Loop {
    int kernel = 0;
    int ndim = 2;
    int lo[3] = {0, 0, 0};
    int hi[3] = {1, 1, 1};
    std::vector<Arg> args;
    std::vector<double> params;
    long long points() const {
        long long n = 1;
        for (int a = 0; a < ndim; ++a) n *= (long long)(hi[a] > lo[a] ? hi[a] - lo[a] : 0);
        return n;
    }
};

// Tile t moves slow rows [a, b). x0 == x1: whole rows. x0 < x1: the rows were first
// written over x in [x0, x1) (all other non-slow axes complete), so only the columns
// outside [x0, x1) -- the halo the writer leaves alone -- are copied.
struct Interval { int t, a, b, x0 = 0, x1 = 0; };

struct DatPlan {
    int dat = -1;
    bool resident = false;     // kept whole in device memory across chains: no copies
    int S = 0;                 // slab rows; row y lives at slot (y - y0) mod S
    int y0 = 0, nrows = 0;
    long long off = 0;         // arena byte offset of the slab (resident: of the dataset)
    std::vector<Interval> up, down;
    std::vector<int> first, last;      // per row: first / last tile touching it, -1 if none
    std::vector<uint8_t> need_up, dl;  // per row: uploaded (1 whole, 2 columns) / downloaded
    std::vector<int> wx0, wx1;         // per row with need_up == 2: x range of its first writer
};

struct RedPlan {
    int handle = -1;
    int op = 0;
    long long part_off = 0;   // arena byte offset of this handle's partials
    long long count = 0;      // number of partials (doubles)
};

// Datasets a streamed plan keeps resident: arena offset per dataset handle (-1 for a
// streamed dataset), inside a region of `bytes` at the start of the arena, and the share of
// the budget the region may take (the planner's residency level).
struct Residency {
    std::vector<long long> off;
    long long bytes = 0;
    double level = 0.0;
    bool any() const { return bytes > 0; }
};

struct Plan {
    uint64_t sig = 0;
    bool valid = false;
    int T = 1, h = 0, depth = 3, L = 0;
    int Y0 = 0, Y1 = 0;
    bool incore = false;
    std::vector<int> se;                 // (t * L + i) * 2 + {0, 1}
    std::vector<DatPlan> dp;
    std::vector<int> dat_index;          // dataset handle -> index in dp (or -1)
    std::vector<RedPlan> rp;
    // Scratch offsets below are relative to the first byte after the slabs (or after
    // the resident datasets in in-core mode).
    std::vector<long long> loop_part;    // per loop: offset of its partials (or -1)
    std::vector<int> loop_chunks;        // per loop: partial chunks per slow row
    std::vector<int> loop_red;           // per loop: index into rp (or -1)
    std::vector<int> loop_param;         // per loop: offset (doubles) into the parameter block
    int nparams = 0;
    long long params_off = 0, paramsf_off = 0, results_off = 0;
    long long slab_bytes = 0;            // end of the slabs (resident region included)
    long long res_bytes = 0;             // resident region at the start of the arena
    int res_dats = 0;                    // datasets kept resident
    double res_level = 0.0;
    long long scratch_bytes = 0;         // partials + parameters + results
    long long arena_bytes = 0;           // slab_bytes + scratch_bytes
    int s(int t, int i) const { return se[((size_t)t * L + i) * 2]; }
    int e(int t, int i) const { return se[((size_t)t * L + i) * 2 + 1]; }
};

// Points per reduction partial along the flattened non-slow axes of a row.
constexpr long long kRedChunk = 4096;

long long align_up(long long v, long long a);

// Analysis (analysis.cpp). Returns false with `err` set if the chain is invalid.
uint64_t chain_signature(const std::vector<Loop>& loops, const std::vector<Dat>& dats,
                         uint32_t flags);
bool build_plan(const std::vector<Loop>& loops, const std::vector<Dat>& dats,
                const std::vector<int>& red_ops, int h, int depth, uint32_t flags,
                bool incore, Plan& plan, std::string& err, const Residency* res = nullptr);
// Largest tile height (>= 1) whose plan fits `budget` bytes; 0 if none fits.
int fit_tile_height(const std::vector<Loop>& loops, const std::vector<Dat>& dats,
                    const std::vector<int>& red_ops, int depth, uint32_t flags,
                    long long budget, std::string& err, const Residency* res = nullptr);
// Residency of a streamed chain at `level` (share of the budget for resident datasets):
// the datasets the chain moves most bytes for per byte they occupy (uploads plus
// downloads of one chain, from a plan without residency), taken greedily while they fit.
Residency choose_residency(const std::vector<Loop>& loops, const std::vector<Dat>& dats,
                           const std::vector<int>& red_ops, uint32_t flags, long long budget,
                           double level);
bool full_row_write(const Loop& lp, const Dat& d);

}  // namespace oc
