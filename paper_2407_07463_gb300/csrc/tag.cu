// Occupancy bits, near-contact test, tagging and tagged near-contact pairs
// (Section 2.3, Steps 1-3; tag.h).
//
// Occupancy of every field is packed one bit per cell, rows of ceil(nx/32)
// words: Step 1 then reads 1/32 (FP32) or 1/64 (FP64) of the bytes of c and
// tests 32 cells per 32-bit word with shifts and ANDs.  Tagging is a
// union-find over the occupied cells (links always to the smaller index, so
// each component's root is its smallest linear index) followed by a prefix
// sum over the roots, which yields exactly the numbering of a flood fill in
// linear-index order.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace vof {

// --------------------------------------------------------------------------
// occupancy bits

template <typename T>
__global__ void __launch_bounds__(256) k_pack_bits(const T* __restrict__ c, uint32_t* __restrict__ bits,
                                                   Dims g, int K, T tau) {
    long long words = (long long)K * g.rows * g.W;
    int lane = threadIdx.x & 31;
    long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    long long per_field = (long long)g.rows * g.W;
    for (long long wd = warp; wd < words; wd += nwarps) {
        int f = (int)(wd / per_field);
        long long rem = wd - (long long)f * per_field;
        int row = (int)(rem / g.W);
        int w = (int)(rem - (long long)row * g.W);
        int x = w * 32 + lane;
        bool v = x < g.nx && c[(size_t)f * g.N + (size_t)row * g.nx + x] > tau;
        unsigned m = __ballot_sync(0xffffffffu, v);
        if (lane == 0) bits[wd] = m;
    }
}

cudaError_t pack_bits(const void* c, bool fp64, uint32_t* bits, const Dims& g, int K, double tau,
                      cudaStream_t st) {
    long long words = (long long)K * g.rows * g.W;
    int blocks = grid_for(words * 32, 256);
    if (fp64)
        k_pack_bits<double><<<blocks, 256, 0, st>>>((const double*)c, bits, g, K, tau);
    else
        k_pack_bits<float><<<blocks, 256, 0, st>>>((const float*)c, bits, g, K, (float)tau);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Box dilation of bit planes (plane blockIdx.y at blockIdx.y * per-field
// words), one axis per pass, periodic: a cell of dst is set when a cell of
// src within `reach` of it along the pass's axis is.  The three passes give
// the cells within Chebyshev distance `reach` of a set cell.
__global__ void __launch_bounds__(256) k_dilate_x(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst,
                                                  Dims g, int reach) {
    const long long pf = (long long)g.rows * g.W;
    src += (size_t)blockIdx.y * pf;
    dst += (size_t)blockIdx.y * pf;
    const bool aligned = (g.nx & 31) == 0;
    const uint32_t tail = (g.nx & 31) ? (1u << (g.nx & 31)) - 1u : 0xffffffffu;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < pf;
         w += (long long)gridDim.x * blockDim.x) {
        const int row = (int)w / g.W, wi = (int)w - row * g.W;
        const uint32_t* r = src + (size_t)row * g.W;
        uint32_t acc = 0u;
        if (aligned) {
            const uint32_t l = r[wi == 0 ? g.W - 1 : wi - 1], c = r[wi], h = r[wi + 1 == g.W ? 0 : wi + 1];
            if (l | c | h)
                for (int dx = -reach; dx <= reach; ++dx) acc |= shift_window(l, c, h, dx);
        } else {
            for (int dx = -reach; dx <= reach; ++dx) acc |= row_window(r, g.W, g.nx, wi * 32 + dx);
            if (wi == g.W - 1) acc &= tail;
        }
        dst[w] = acc;
    }
}

// axis 1: along y, axis 2: along z
__global__ void __launch_bounds__(256) k_dilate_rows(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst,
                                                     Dims g, int reach, int axis) {
    const long long pf = (long long)g.rows * g.W;
    src += (size_t)blockIdx.y * pf;
    dst += (size_t)blockIdx.y * pf;
    const bool near = reach < (axis == 1 ? g.ny : g.nz);
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < pf;
         w += (long long)gridDim.x * blockDim.x) {
        const int row = (int)w / g.W, wi = (int)w - row * g.W;
        const int k = row / g.ny, j = row - k * g.ny;
        uint32_t acc = 0u;
        for (int dd = -reach; dd <= reach; ++dd) {
            const int rr = axis == 1 ? k * g.ny + (near ? wrap1(j + dd, g.ny) : wrapi(j + dd, g.ny))
                                     : (near ? wrap1(k + dd, g.nz) : wrapi(k + dd, g.nz)) * g.ny + j;
            acc |= src[(size_t)rr * g.W + wi];
        }
        dst[w] = acc;
    }
}

cudaError_t dilate_planes(const uint32_t* src, uint32_t* dst, uint32_t* tmp, int n, const Dims& g, int reach,
                          cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const long long pf = (long long)g.rows * g.W;
    const dim3 grid(grid_for(pf, 256, std::max(1, sm_count() * 32 / n)), n);
    k_dilate_x<<<grid, 256, 0, st>>>(src, dst, g, reach);
    k_dilate_rows<<<grid, 256, 0, st>>>(dst, tmp, g, reach, 1);
    k_dilate_rows<<<grid, 256, 0, st>>>(tmp, dst, g, reach, 2);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Step 1: near contact.  For every cell with c <= tau, is there an offset
// delta in [-w,w]^3 \ {0} with both cells x + delta and x - delta occupied?
// One offset per opposite pair: the first nonzero of (dz, dy, dx) positive.

__global__ void __launch_bounds__(256) k_near_contact(const uint32_t* __restrict__ bits,
                                                      uint32_t* __restrict__ ncmap,
                                                      int* __restrict__ flags, Dims g, int K, int w) {
    // one field per blockIdx.y; 32-bit word indices within the field
    const int per_field = g.rows * g.W;
    const int f = blockIdx.y;
    const int stride = gridDim.x * blockDim.x;
    const bool aligned = (g.nx & 31) == 0;
    const bool wide = g.ny > 2 * w && g.nz > 2 * w;
    for (int rem = blockIdx.x * blockDim.x + threadIdx.x; rem < per_field; rem += stride) {
        const size_t idx = (size_t)f * per_field + rem;
        int row = rem / g.W;
        int wi = rem - row * g.W;
        int j = row % g.ny, k = row / g.ny;
        const uint32_t* fb = bits + (size_t)f * per_field;
        uint32_t centre = fb[(size_t)row * g.W + wi];
        uint32_t valid = (wi == g.W - 1 && (g.nx & 31)) ? ((1u << (g.nx & 31)) - 1u) : 0xffffffffu;
        uint32_t empty = ~centre & valid;
        uint32_t acc = 0;
        int x0 = wi * 32;
        int wl = wi == 0 ? g.W - 1 : wi - 1, wr = wi + 1 == g.W ? 0 : wi + 1;
        if (empty) {
            for (int dz = 0; dz <= w && (acc & empty) != empty; ++dz) {
                int ka, kb;
                if (wide) {
                    ka = k + dz; if (ka >= g.nz) ka -= g.nz;
                    kb = k - dz; if (kb < 0) kb += g.nz;
                } else {
                    ka = wrapi(k + dz, g.nz);
                    kb = wrapi(k - dz, g.nz);
                }
                for (int dy = (dz == 0 ? 0 : -w); dy <= w; ++dy) {
                    int ja, jb;
                    if (wide) {
                        ja = j + dy; if (ja >= g.ny) ja -= g.ny; else if (ja < 0) ja += g.ny;
                        jb = j - dy; if (jb >= g.ny) jb -= g.ny; else if (jb < 0) jb += g.ny;
                    } else {
                        ja = wrapi(j + dy, g.ny);
                        jb = wrapi(j - dy, g.ny);
                    }
                    const uint32_t* ra = fb + (size_t)(ka * g.ny + ja) * g.W;
                    const uint32_t* rb = fb + (size_t)(kb * g.ny + jb) * g.W;
                    int dx0 = (dz == 0 && dy == 0) ? 1 : -w;
                    if (aligned) {
                        uint32_t al = ra[wl], ac = ra[wi], ar = ra[wr];
                        uint32_t bl = rb[wl], bc = rb[wi], br = rb[wr];
                        if (((al | ac | ar) == 0) || ((bl | bc | br) == 0)) continue;
                        for (int dx = dx0; dx <= w; ++dx)
                            acc |= shift_window(al, ac, ar, dx) & shift_window(bl, bc, br, -dx);
                    } else {
                        for (int dx = dx0; dx <= w; ++dx)
                            acc |= row_window(ra, g.W, g.nx, x0 + dx) & row_window(rb, g.W, g.nx, x0 - dx);
                    }
                }
            }
        }
        uint32_t res = acc & empty;
        if (ncmap) ncmap[idx] = res;
        // one atomic per field once it is flagged, not one per word: bit 0
        // Step 1 fired, bit 1 the field holds an occupied cell
        if (res && (*(volatile int*)&flags[f] & 1) == 0) atomicOr(&flags[f], 1);
        if ((centre & valid) && (*(volatile int*)&flags[f] & 2) == 0) atomicOr(&flags[f], 2);
    }
}

// The same test on tiles of whole rows, for rows of a power-of-two number
// W <= 32 of whole words: a block of 256 threads takes 256 / W rows of one
// field (TY = 2^ty_log along y by TZ along z, one word per thread), stages
// them with a halo of w rows along y and z in shared memory, and reads every
// neighbour row from there.
constexpr int kNcThreads = 256;
__global__ void __launch_bounds__(kNcThreads) k_near_contact_tile(const uint32_t* __restrict__ bits,
                                                                  uint32_t* __restrict__ ncmap,
                                                                  int* __restrict__ flags, Dims g, int w, int lw,
                                                                  int ty_log, int tiles_y) {
    extern __shared__ uint32_t s_rows[];
    const int f = blockIdx.y;
    const int W = 1 << lw;
    const int TY = 1 << ty_log, TZ = (kNcThreads >> lw) >> ty_log;
    const int HY = TY + 2 * w, HZ = TZ + 2 * w;
    const int tz = blockIdx.x / tiles_y, tyi = blockIdx.x - tz * tiles_y;
    const int j0 = tyi * TY, k0 = tz * TZ;
    const size_t per_field = (size_t)g.rows * W;
    const uint32_t* fb = bits + (size_t)f * per_field;
    // the tile's rows and their halo (the caller ensures TY + w <= ny and
    // TZ + w <= nz, so every staged index is within one period)
    uint32_t any = 0u;
    for (int t = threadIdx.x; t < HY * HZ * W; t += kNcThreads) {
        const int wi = t & (W - 1), r = t >> lw;
        const int hz = r / HY, hy = r - hz * HY;
        const int j = wrap1(j0 - w + hy, g.ny), k = wrap1(k0 - w + hz, g.nz);
        const uint32_t v = fb[(size_t)(k * g.ny + j) * W + wi];
        s_rows[t] = v;
        any |= v;
    }
    const bool occupied = __syncthreads_or(any != 0u);
    const int wi = threadIdx.x & (W - 1), r = threadIdx.x >> lw;
    const int lz = r >> ty_log, ly = r - (lz << ty_log);
    const int j = j0 + ly, k = k0 + lz;
    if (j >= g.ny || k >= g.nz) return;  // a partial tile at the grid's end
    if (!occupied) {  // tile and halo empty: nothing fires, nothing is occupied
        if (ncmap) ncmap[(size_t)f * per_field + (size_t)(k * g.ny + j) * W + wi] = 0u;
        return;
    }
    const uint32_t* base = s_rows + ((size_t)(lz + w) * HY + (ly + w)) * W;
    const uint32_t centre = base[wi];
    const uint32_t empty = ~centre;
    const int wl = (wi - 1) & (W - 1), wr = (wi + 1) & (W - 1);
    uint32_t acc = 0;
    if (empty) {
        for (int dz = 0; dz <= w && (acc & empty) != empty; ++dz) {
            for (int dy = (dz == 0 ? 0 : -w); dy <= w; ++dy) {
                const uint32_t* ra = base + (dz * HY + dy) * W;
                const uint32_t* rb = base - (dz * HY + dy) * W;
                const uint32_t al = ra[wl], ac = ra[wi], ar = ra[wr];
                const uint32_t bl = rb[wl], bc = rb[wi], br = rb[wr];
                if (((al | ac | ar) == 0) || ((bl | bc | br) == 0)) continue;
                for (int dx = (dz == 0 && dy == 0) ? 1 : -w; dx <= w; ++dx)
                    acc |= shift_window(al, ac, ar, dx) & shift_window(bl, bc, br, -dx);
            }
        }
    }
    const uint32_t res = acc & empty;
    if (ncmap) ncmap[(size_t)f * per_field + (size_t)(k * g.ny + j) * W + wi] = res;
    if (res && (*(volatile int*)&flags[f] & 1) == 0) atomicOr(&flags[f], 1);
    if (centre && (*(volatile int*)&flags[f] & 2) == 0) atomicOr(&flags[f], 2);
}

cudaError_t near_contact(const uint32_t* bits, uint32_t* ncmap, int* flags, const Dims& g, int K, int w,
                         cudaStream_t st) {
    if (K <= 0) return cudaSuccess;
    const long long per_field = (long long)g.rows * g.W;
    int lw = 0;
    while ((1 << lw) < g.W) ++lw;
    const int R = kNcThreads >> lw;  // rows per tile
    int ty_log = 0;
    while ((1 << (2 * (ty_log + 1))) <= R) ++ty_log;  // TY ~ sqrt(R)
    const int TY = 1 << ty_log, TZ = R / TY;
    const bool tiled = (g.nx & 31) == 0 && (1 << lw) == g.W && g.W <= 32 && w >= 1 && w <= 4 && TY + w <= g.ny &&
                       TZ + w <= g.nz && w < g.ny && w < g.nz;
    if (tiled) {
        const int tiles_y = (g.ny + TY - 1) / TY, tiles_z = (g.nz + TZ - 1) / TZ;
        const size_t smem = (size_t)(TY + 2 * w) * (TZ + 2 * w) * g.W * sizeof(uint32_t);
        k_near_contact_tile<<<dim3(tiles_y * tiles_z, K), kNcThreads, smem, st>>>(bits, ncmap, flags, g, w, lw, ty_log,
                                                                                 tiles_y);
    } else {
        k_near_contact<<<dim3(grid_for(per_field, 256, sm_count() * 32 / K + 1), K), 256, 0, st>>>(bits, ncmap, flags,
                                                                                                   g, K, w);
    }
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Tagging (connected components, periodic)
//
// Union-find over occupied cells; every link points to a smaller linear
// index, so a component's root is its smallest cell.  6-connectivity works
// on runs of the occupancy bits: within a row each cell links to the start
// of its run (or to the last cell of the previous word when the run crosses
// a word), and rows are joined by one union per maximal segment where a row
// and its -y / -z neighbour row are both occupied.  26-connectivity uses one
// union per occupied neighbour pair.  Empty cells never touch `parent`.

__device__ __forceinline__ int find_root(const int* parent, int x) {
    int p = __ldcg(parent + x);
    while (p != x) {
        x = p;
        p = __ldcg(parent + x);
    }
    return x;
}

__device__ __forceinline__ void unite(int* parent, int a, int b) {
    while (true) {
        a = find_root(parent, a);
        b = find_root(parent, b);
        if (a == b) return;
        if (a < b) {
            int t = a;
            a = b;
            b = t;
        }
        int old = atomicMin(parent + a, b);
        if (old == a) return;
        a = old;
    }
}

// The labelling kernels run one slot of a LabelSlots per blockIdx.y: the
// slot's field selects the bit plane (and the labels), the slot itself the
// scratch (parent and rank arrays, block totals and offsets).
__device__ __forceinline__ const uint32_t* slot_bits(const uint32_t* bits, const LabelSlots& ls, const Dims& g) {
    return bits + (size_t)ls.f[blockIdx.y] * ((size_t)g.rows * g.W);
}
__host__ __device__ __forceinline__ int label_blocks(const Dims& g) { return (g.N + 1023) / 1024; }

// Heads of the runs of a row word w: the run starts, plus bit 0 where a run
// continues from the row's previous word (carry: that word's last bit).
__device__ __forceinline__ uint32_t run_starts(uint32_t w, uint32_t carry) { return w & ~((w << 1) | carry); }
__device__ __forceinline__ uint32_t run_heads(uint32_t w, uint32_t carry) { return run_starts(w, carry) | (w & carry); }
// The head of the run holding bit b of a word with heads h.
__device__ __forceinline__ int head_of(uint32_t h, int b) {
    return 31 - __clz(h & (b == 31 ? 0xffffffffu : ((2u << b) - 1u)));
}

// Heads of the runs of word wi of a row (cells of whole words) whose word
// is w: the carry is the previous word's last bit.
__device__ __forceinline__ uint32_t word_heads(const uint32_t* row_bits, int wi, uint32_t w) {
    return run_heads(w, wi > 0 ? (row_bits[wi - 1] >> 31) : 0u);
}

// HEADS (rows of whole words): only the heads of runs get a link -- a run
// start links to itself, and a run continuing from the previous word links
// its bit 0 to the head of that word's last run; the other cells are never
// read.  Otherwise every occupied cell links to its run's start (or to the
// previous word's last cell).
template <bool HEADS>
__global__ void k_ccl_init_runs(const uint32_t* __restrict__ bits, int* __restrict__ parent, Dims g,
                                const __grid_constant__ LabelSlots ls) {
    const uint32_t* bits_f = slot_bits(bits, ls, g);
    parent += (size_t)blockIdx.y * g.N;
    const long long words = (long long)g.rows * g.W;
    for (long long gw = (long long)blockIdx.x * blockDim.x + threadIdx.x; gw < words;
         gw += (long long)gridDim.x * blockDim.x) {
        const uint32_t w = bits_f[gw];
        if (!w) continue;
        const int row = (int)gw / g.W, wi = (int)gw - row * g.W;
        const uint32_t carry = wi > 0 ? (bits_f[gw - 1] >> 31) : 0u;
        const uint32_t starts = w & ~((w << 1) | carry);
        const int x0 = row * g.nx + wi * 32;
        if (HEADS) {
            uint32_t m = starts;
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1u;
                parent[x0 + b] = x0 + b;
            }
            if (w & carry)
                parent[x0] = x0 - 32 + head_of(word_heads(bits_f + (size_t)row * g.W, wi - 1, bits_f[gw - 1]), 31);
            continue;
        }
        uint32_t m = w;
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1u;
            const uint32_t below = starts & (b == 31 ? 0xffffffffu : ((2u << b) - 1u));
            parent[x0 + b] = below ? x0 + (31 - __clz(below)) : x0 - 1;
        }
    }
}

// one union per maximal overlap segment of row `w` with neighbour row `wn`
__device__ __forceinline__ void join_rows(int* parent, uint32_t w, uint32_t wn, uint32_t carry, int x0, int xn0) {
    const uint32_t ov = w & wn;
    uint32_t seg = ov & ~((ov << 1) | carry);
    while (seg) {
        const int b = __ffs(seg) - 1;
        seg &= seg - 1u;
        unite(parent, x0 + b, xn0 + b);
    }
}

// HEADS: the unions join the heads of the runs holding the overlap's first
// cell in either row.
template <bool HEADS>
__global__ void k_ccl_merge_runs(const uint32_t* __restrict__ bits, int* parent, Dims g,
                                 const __grid_constant__ LabelSlots ls) {
    const uint32_t* bits_f = slot_bits(bits, ls, g);
    parent += (size_t)blockIdx.y * g.N;
    const long long words = (long long)g.rows * g.W;
    for (long long gw = (long long)blockIdx.x * blockDim.x + threadIdx.x; gw < words;
         gw += (long long)gridDim.x * blockDim.x) {
        const uint32_t w = bits_f[gw];
        if (!w) continue;
        const int row = (int)gw / g.W, wi = (int)gw - row * g.W;
        const int j = row % g.ny, k = row / g.ny;
        const int x0 = row * g.nx + wi * 32;
        const uint32_t* rb = bits_f + (size_t)row * g.W;
        const uint32_t hw = HEADS ? word_heads(rb, wi, w) : 0u;
        if (wi == 0 && (w & 1u) && g.nx > 1) {
            const int last = g.nx - 1;
            const uint32_t wl = rb[last >> 5];
            if ((wl >> (last & 31)) & 1u) {
                const int xl = HEADS ? row * g.nx + (last & ~31) + head_of(word_heads(rb, last >> 5, wl), last & 31)
                                     : x0 + last;
                unite(parent, x0, xl);
            }
        }
        const int rows_nb[2] = {k * g.ny + (j == 0 ? g.ny - 1 : j - 1), (k == 0 ? g.nz - 1 : k - 1) * g.ny + j};
        for (int q = 0; q < 2; ++q) {
            const int rn = rows_nb[q];
            if (rn == row) continue;
            const size_t gn = (size_t)rn * g.W + wi;
            const uint32_t wn = bits_f[gn];
            const uint32_t carry = wi > 0 ? ((bits_f[gw - 1] & bits_f[gn - 1]) >> 31) : 0u;
            if (!HEADS) {
                join_rows(parent, w, wn, carry, x0, rn * g.nx + wi * 32);
                continue;
            }
            const uint32_t ov = w & wn;
            uint32_t seg = ov & ~((ov << 1) | carry);
            if (!seg) continue;
            const uint32_t hn = word_heads(bits_f + (size_t)rn * g.W, wi, wn);
            const int xn0 = rn * g.nx + wi * 32;
            while (seg) {
                const int b = __ffs(seg) - 1;
                seg &= seg - 1u;
                unite(parent, x0 + head_of(hw, b), xn0 + head_of(hn, b));
            }
        }
    }
}

__global__ void k_ccl_init(const uint32_t* __restrict__ bits, int* __restrict__ parent, Dims g, const __grid_constant__ LabelSlots ls) {
    const uint32_t* bits_f = slot_bits(bits, ls, g);
    parent += (size_t)blockIdx.y * g.N;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < g.N; x += gridDim.x * blockDim.x) {
        int i = x % g.nx, row = x / g.nx;
        if (bit_at(bits_f, g.W, row, i)) parent[x] = x;
    }
}

__global__ void k_ccl_merge26(const uint32_t* __restrict__ bits, int* parent, Dims g, const __grid_constant__ LabelSlots ls) {
    const uint32_t* bits_f = slot_bits(bits, ls, g);
    parent += (size_t)blockIdx.y * g.N;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < g.N; x += gridDim.x * blockDim.x) {
        int i, j, k;
        decode(x, g, i, j, k);
        if (!bit_at(bits_f, g.W, k * g.ny + j, i)) continue;
        for (int dz = -1; dz <= 0; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    bool back = dz < 0 || (dz == 0 && (dy < 0 || (dy == 0 && dx < 0)));
                    if (!back) continue;
                    int ii = wrapi(i + dx, g.nx), jj = wrapi(j + dy, g.ny), kk = wrapi(k + dz, g.nz);
                    if (!bit_at(bits_f, g.W, kk * g.ny + jj, ii)) continue;
                    unite(parent, x, cell(ii, jj, kk, g));
                }
    }
}

__global__ void k_ccl_flatten(const uint32_t* __restrict__ bits, int* parent, Dims g, const __grid_constant__ LabelSlots ls) {
    const uint32_t* bits_f = slot_bits(bits, ls, g);
    parent += (size_t)blockIdx.y * g.N;
    const long long words = (long long)g.rows * g.W;
    for (long long gw = (long long)blockIdx.x * blockDim.x + threadIdx.x; gw < words;
         gw += (long long)gridDim.x * blockDim.x) {
        uint32_t m = bits_f[gw];
        if (!m) continue;
        const int row = (int)gw / g.W, wi = (int)gw - row * g.W;
        const int x0 = row * g.nx + wi * 32;
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1u;
            parent[x0 + b] = find_root(parent, x0 + b);
        }
    }
}

// Flattening for the run-based links of 6-connectivity: only the head of
// every run of every word takes its root (a run's other cells link to their
// head, or to the previous word, and are labelled through their head).
__global__ void k_ccl_flatten_runs(const uint32_t* __restrict__ bits, int* parent, Dims g,
                                   const __grid_constant__ LabelSlots ls) {
    const uint32_t* bits_f = slot_bits(bits, ls, g);
    parent += (size_t)blockIdx.y * g.N;
    const long long words = (long long)g.rows * g.W;
    for (long long gw = (long long)blockIdx.x * blockDim.x + threadIdx.x; gw < words;
         gw += (long long)gridDim.x * blockDim.x) {
        const uint32_t w = bits_f[gw];
        if (!w) continue;
        const int row = (int)gw / g.W, wi = (int)gw - row * g.W;
        const uint32_t carry = wi > 0 ? (bits_f[gw - 1] >> 31) : 0u;
        uint32_t h = run_heads(w, carry);
        const int x0 = row * g.nx + wi * 32;
        while (h) {
            const int b = __ffs(h) - 1;
            h &= h - 1u;
            parent[x0 + b] = find_root(parent, x0 + b);
        }
    }
}

// Per block of 1024 cells: rank of each root among the block's roots.
__global__ void __launch_bounds__(1024) k_ccl_count(const uint32_t* __restrict__ bits,
                                                    const int* __restrict__ parent, int* __restrict__ rank,
                                                    int* __restrict__ block_tot, Dims g, const __grid_constant__ LabelSlots ls) {
    const uint32_t* bits_f = slot_bits(bits, ls, g);
    parent += (size_t)blockIdx.y * g.N;
    rank += (size_t)blockIdx.y * g.N;
    block_tot += (size_t)blockIdx.y * (label_blocks(g) + 1);
    __shared__ int warp_tot[32];
    int x = blockIdx.x * 1024 + threadIdx.x;
    bool root = false;
    if (x < g.N) {
        int i = x % g.nx, row = x / g.nx;
        root = bit_at(bits_f, g.W, row, i) && parent[x] == x;
    }
    unsigned m = __ballot_sync(0xffffffffu, root);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_tot[wid] = __popc(m);
    __syncthreads();
    if (wid == 0) {
        int v = warp_tot[lane];
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        warp_tot[lane] = incl - v;
        if (lane == 31) block_tot[blockIdx.x] = incl;
    }
    __syncthreads();
    if (root) rank[x] = warp_tot[wid] + __popc(m & ((1u << lane) - 1u));
}

// The same for rows of whole 32-cell words (bit word gw holds cells
// 32 gw .. 32 gw + 31): one warp per 1024-cell block, a lane per word, and
// only the occupied cells read their parent.
// RUNS: the run-based links of 6-connectivity, where only run starts can be
// roots.
template <bool RUNS>
__global__ void __launch_bounds__(256) k_ccl_count_words(const uint32_t* __restrict__ bits,
                                                         const int* __restrict__ parent, int* __restrict__ rank,
                                                         int* __restrict__ block_tot, int nblk, Dims g, const __grid_constant__ LabelSlots ls) {
    const long long words = (long long)g.rows * g.W;
    const uint32_t* bits_f = slot_bits(bits, ls, g);
    parent += (size_t)blockIdx.y * g.N;
    rank += (size_t)blockIdx.y * g.N;
    block_tot += (size_t)blockIdx.y * (nblk + 1);
    const int lane = threadIdx.x & 31;
    const int rb = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (rb >= nblk) return;  // whole warps leave together
    const long long gw = (long long)rb * 32 + lane;
    uint32_t m = gw < words ? bits_f[gw] : 0u, rm = 0u;
    const int x0 = (int)(gw * 32);
    if (RUNS && m) m = run_starts(m, ((int)gw % g.W) ? (bits_f[gw - 1] >> 31) : 0u);
    while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1u;
        if (parent[x0 + b] == x0 + b) rm |= 1u << b;
    }
    const int cnt = __popc(rm);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) block_tot[rb] = incl;
    int r = incl - cnt;
    while (rm) {
        const int b = __ffs(rm) - 1;
        rm &= rm - 1u;
        rank[x0 + b] = r++;
    }
}

// Exclusive scan of n block totals by one block of 1024 threads; off[n] =
// total.
__device__ void scan_block(const int* __restrict__ tot, int* __restrict__ off, int n, int* total_out) {
    __shared__ int wsum[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < n; base += 1024) {
        int i = base + threadIdx.x;
        int v = i < n ? tot[i] : 0;
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int s = wsum[lane];
            int si = s;
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(0xffffffffu, si, o);
                if (lane >= o) si += t;
            }
            wsum[lane] = si - s;
        }
        __syncthreads();
        int excl = carry + wsum[wid] + incl - v;
        if (i < n) off[i] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        off[n] = carry;
        if (total_out) *total_out = carry;
    }
}

__global__ void __launch_bounds__(1024) k_scan_blocks(const int* __restrict__ tot, int* __restrict__ off, int n,
                                                      int* total_out) {
    scan_block(tot, off, n, total_out);
}

// One block per slot (blockIdx.y): the slot's block totals into its offsets,
// the total (the field's tag count) into n_out[field].
__global__ void __launch_bounds__(1024) k_scan_label(const int* __restrict__ tot, int* __restrict__ off, int nb,
                                                     int* n_out, const __grid_constant__ LabelSlots ls) {
    const size_t o = (size_t)blockIdx.y * (nb + 1);
    scan_block(tot + o, off + o, nb, n_out ? n_out + ls.f[blockIdx.y] : nullptr);
}

cudaError_t scan_counts(const int* counts, int* off, int n, cudaStream_t st) {
    k_scan_blocks<<<1, 1024, 0, st>>>(counts, off, n, nullptr);
    return cudaGetLastError();
}

// Exclusive scan of the face-list segment lengths, then the segment holding
// the first entry of every tile of kFaceTile consecutive entries:
// tile_seg[t] = s with off[s] <= t * kFaceTile < off[s + 1] (at most
// tile_cap tiles are recorded).
__global__ void __launch_bounds__(1024) k_scan_faces(const int* __restrict__ counts, int* __restrict__ off, int n,
                                                     int* __restrict__ tile_seg, int tile_cap) {
    __shared__ int wsum[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < n; base += 1024) {
        const int i = base + threadIdx.x;
        const int v = i < n ? counts[i] : 0;
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const int s0 = wsum[lane];
            int si = s0;
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, si, o);
                if (lane >= o) si += t;
            }
            wsum[lane] = si - s0;
        }
        __syncthreads();
        const int excl = carry + wsum[wid] + incl - v;
        if (i < n) {
            off[i] = excl;
            // tiles whose first entry lies in this segment
            const int t0 = (excl + kFaceTile - 1) / kFaceTile;
            const int t1 = min((excl + v + kFaceTile - 1) / kFaceTile, tile_cap);
            for (int t = t0; t < t1; ++t) tile_seg[t] = i;
        }
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) off[n] = carry;
}

cudaError_t scan_face_counts(const int* counts, int* off, int n, int* tile_seg, int tile_cap, cudaStream_t st) {
    k_scan_faces<<<1, 1024, 0, st>>>(counts, off, n, tile_seg, tile_cap);
    return cudaGetLastError();
}

// Labels for rows of whole 32-cell words: a thread per word writes its 32
// labels as eight 16-byte stores; occupied cells take 1 + the global rank
// of their root.
// RUNS: run-based links, where a cell's root is that of its run's head.
// SPARSE: words without an occupied cell are not written (their labels are
// left as they were), for callers that read labels only at occupied cells.
template <bool RUNS, bool SPARSE>
__global__ void __launch_bounds__(256) k_ccl_relabel_words(const uint32_t* __restrict__ bits,
                                                           const int* __restrict__ parent,
                                                           const int* __restrict__ rank, const int* __restrict__ off,
                                                           int* __restrict__ label, int* __restrict__ root_of,
                                                           int root_cap, Dims g, const __grid_constant__ LabelSlots ls) {
    const long long words = (long long)g.rows * g.W;
    const uint32_t* bits_f = slot_bits(bits, ls, g);
    parent += (size_t)blockIdx.y * g.N;
    rank += (size_t)blockIdx.y * g.N;
    off += (size_t)blockIdx.y * (label_blocks(g) + 1);
    label += (size_t)ls.f[blockIdx.y] * g.N;
    for (long long gw = (long long)blockIdx.x * blockDim.x + threadIdx.x; gw < words;
         gw += (long long)gridDim.x * blockDim.x) {
        const uint32_t w = bits_f[gw];
        if (SPARSE && !w) continue;
        const int x0 = (int)(gw * 32);
        int4* dst = reinterpret_cast<int4*>(label + x0);
        uint32_t heads = 0u;
        if (RUNS && w) heads = run_heads(w, ((int)gw % g.W) ? (bits_f[gw - 1] >> 31) : 0u);
        int last_head = -1, last_l = 0;  // the cells of a run share their head's tag
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            int l4[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int b = 4 * q + e;
                int l = 0;
                if ((w >> b) & 1u) {
                    const int x = x0 + b;
                    if (RUNS) {
                        const int h = head_of(heads, b);
                        if (h != last_head) {
                            const int r = parent[x0 + h];
                            last_l = off[r >> 10] + rank[r] + 1;
                            last_head = h;
                            if (r == x && root_of && last_l <= root_cap) root_of[last_l - 1] = x;
                        }
                        l = last_l;
                    } else {
                        const int r = parent[x];
                        l = off[r >> 10] + rank[r] + 1;
                        if (r == x && root_of && l <= root_cap) root_of[l - 1] = x;
                    }
                }
                l4[e] = l;
            }
            dst[q] = make_int4(l4[0], l4[1], l4[2], l4[3]);
        }
    }
}

// Labels of one row segment per warp: 0 for empty cells, 1 + rank of the
// root for occupied ones.
__global__ void k_ccl_relabel(const uint32_t* __restrict__ bits, const int* __restrict__ parent,
                              const int* __restrict__ rank, const int* __restrict__ off, int* __restrict__ label,
                              int* __restrict__ root_of, int root_cap, Dims g, const __grid_constant__ LabelSlots ls) {
    const uint32_t* bits_f = slot_bits(bits, ls, g);
    parent += (size_t)blockIdx.y * g.N;
    rank += (size_t)blockIdx.y * g.N;
    off += (size_t)blockIdx.y * (label_blocks(g) + 1);
    label += (size_t)ls.f[blockIdx.y] * g.N;
    const int lane = threadIdx.x & 31;
    const long long words = (long long)g.rows * g.W;
    for (long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; gw < words;
         gw += ((long long)gridDim.x * blockDim.x) >> 5) {
        const int row = (int)gw / g.W, wi = (int)gw - row * g.W;
        const int i = wi * 32 + lane;
        if (i >= g.nx) continue;
        const int x = row * g.nx + i;
        int l = 0;
        if ((bits_f[gw] >> lane) & 1u) {
            const int r = parent[x];
            l = off[r >> 10] + rank[r] + 1;
            if (r == x && root_of && l <= root_cap) root_of[l - 1] = x;
        }
        label[x] = l;
    }
}

// The chain of six launches that tags every slot's field; root_of (the
// root cell of tag l at root_of[l - 1], l <= root_cap) only with one slot.
// sparse: labels are needed only at occupied cells.
static cudaError_t label_run(const uint32_t* bits, const Dims& g, int conn, const LabelSlots& ls, int* parent,
                             int* rank, int* block_tot, int* block_off, int* labels, int* root_of, int root_cap,
                             int* n_out, bool sparse, cudaStream_t st, long long* launches) {
    if (ls.n <= 0) return cudaSuccess;
    if (ls.n > kLabelSlots || (root_of && ls.n != 1)) return cudaErrorInvalidValue;
    const int nb = label_blocks(g);
    const long long words = (long long)g.rows * g.W;
    // the slots share the blocks a single field would get
    const int cap = std::max(1, sm_count() * 32 / ls.n);
    const dim3 bw(grid_for(words, 256, cap), ls.n), bc(grid_for(g.N, 256, cap), ls.n);
    // rows of whole words (and a 16-byte-aligned label array): word-wise
    // passes; with 6-connectivity there the union-find links only the heads
    // of runs, and only they are flattened
    const bool wordwise = (g.nx & 31) == 0 && ((uintptr_t)labels & 15) == 0;
    const bool runs = wordwise && conn == 6;
    if (conn == 6) {
        if (runs) {
            k_ccl_init_runs<true><<<bw, 256, 0, st>>>(bits, parent, g, ls);
            k_ccl_merge_runs<true><<<bw, 256, 0, st>>>(bits, parent, g, ls);
        } else {
            k_ccl_init_runs<false><<<bw, 256, 0, st>>>(bits, parent, g, ls);
            k_ccl_merge_runs<false><<<bw, 256, 0, st>>>(bits, parent, g, ls);
        }
    } else {
        k_ccl_init<<<bc, 256, 0, st>>>(bits, parent, g, ls);
        k_ccl_merge26<<<bc, 256, 0, st>>>(bits, parent, g, ls);
    }
    if (runs)
        k_ccl_flatten_runs<<<bw, 256, 0, st>>>(bits, parent, g, ls);
    else
        k_ccl_flatten<<<bw, 256, 0, st>>>(bits, parent, g, ls);
    const dim3 bcnt((nb + 7) / 8, ls.n);
    if (runs)
        k_ccl_count_words<true><<<bcnt, 256, 0, st>>>(bits, parent, rank, block_tot, nb, g, ls);
    else if (wordwise)
        k_ccl_count_words<false><<<bcnt, 256, 0, st>>>(bits, parent, rank, block_tot, nb, g, ls);
    else
        k_ccl_count<<<dim3(nb, ls.n), 1024, 0, st>>>(bits, parent, rank, block_tot, g, ls);
    k_scan_label<<<dim3(1, ls.n), 1024, 0, st>>>(block_tot, block_off, nb, n_out, ls);
    if (runs && sparse)
        k_ccl_relabel_words<true, true><<<bw, 256, 0, st>>>(bits, parent, rank, block_off, labels, root_of, root_cap,
                                                             g, ls);
    else if (runs)
        k_ccl_relabel_words<true, false><<<bw, 256, 0, st>>>(bits, parent, rank, block_off, labels, root_of, root_cap,
                                                              g, ls);
    else if (wordwise)
        k_ccl_relabel_words<false, false><<<bw, 256, 0, st>>>(bits, parent, rank, block_off, labels, root_of,
                                                               root_cap, g, ls);
    else
        k_ccl_relabel<<<dim3(grid_for(words * 32, 256, cap), ls.n), 256, 0, st>>>(bits, parent, rank, block_off,
                                                                                 labels, root_of, root_cap, g, ls);
    if (launches) *launches += 6;
    return cudaGetLastError();
}

cudaError_t label_field(const uint32_t* bits_f, const Dims& g, int conn, int* parent, int* rank,
                        int* block_tot, int* block_off, int* label, int* root_of, int root_cap, int* n_out,
                        cudaStream_t st, long long* launches) {
    LabelSlots one{};
    one.n = 1;
    one.f[0] = 0;
    return label_run(bits_f, g, conn, one, parent, rank, block_tot, block_off, label, root_of, root_cap, n_out, false,
                     st, launches);
}

cudaError_t label_fields(const uint32_t* bits, const Dims& g, int conn, const LabelSlots& ls, int* parent, int* rank,
                         int* block_tot, int* block_off, int* labels, int* n_out, cudaStream_t st,
                         long long* launches) {
    return label_run(bits, g, conn, ls, parent, rank, block_tot, block_off, labels, nullptr, 0, n_out, true, st,
                     launches);
}

// --------------------------------------------------------------------------
// Step 3: distinct tag pairs of opposite occupied cells around near-contact
// cells, deduplicated in an open-addressing set of 64-bit keys
// (field << 60 | lo << 30 | hi).

__device__ __forceinline__ unsigned long long pair_key(int f, int lo, int hi) {
    return ((unsigned long long)f << 60) | ((unsigned long long)lo << 30) | (unsigned long long)hi;
}

__device__ __forceinline__ void set_insert(unsigned long long* table, int mask, unsigned long long key,
                                           int* overflow) {
    unsigned long long h = key * 0x9E3779B97F4A7C15ull;
    int s = (int)(h >> 40) & mask;
    for (int p = 0; p <= mask; ++p) {
        unsigned long long old = atomicCAS(table + s, kEmptyKey, key);
        if (old == kEmptyKey || old == key) return;
        s = (s + 1) & mask;
    }
    atomicExch(overflow, 1);
}

__global__ void k_pairs(const uint32_t* __restrict__ ncmap, const uint32_t* __restrict__ bits,
                        const int* __restrict__ labels, Dims g, int w, unsigned long long* table, int mask,
                        int* overflow, const __grid_constant__ LabelSlots ls) {
    const long long words = (long long)g.rows * g.W;
    const int f = ls.f[blockIdx.y];
    const uint32_t* ncmap_f = ncmap + (size_t)f * words;
    const uint32_t* bits_f = bits + (size_t)f * words;
    const int* label_f = labels + (size_t)f * g.N;
    // offsets of at most w stay within one period of the grid when w < n
    const bool near = w < g.nx && w < g.ny && w < g.nz;
    auto wr = [near](int v, int n) { return near ? wrap1(v, n) : wrapi(v, n); };
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < words;
         idx += (long long)gridDim.x * blockDim.x) {
        uint32_t m = ncmap_f[idx];
        if (!m) continue;
        const int row = (int)idx / g.W, wi = (int)idx - row * g.W;
        const int j = row % g.ny, k = row / g.ny;
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1u;
            const int i = wi * 32 + b;
            for (int dz = 0; dz <= w; ++dz) {
                const int ka = wr(k + dz, g.nz), kb = wr(k - dz, g.nz);
                for (int dy = (dz == 0 ? 0 : -w); dy <= w; ++dy) {
                    const int ja = wr(j + dy, g.ny), jb = wr(j - dy, g.ny);
                    const int ra = ka * g.ny + ja, rb = kb * g.ny + jb;
                    for (int dx = ((dz == 0 && dy == 0) ? 1 : -w); dx <= w; ++dx) {
                        const int ia = wr(i + dx, g.nx), ib = wr(i - dx, g.nx);
                        if (!bit_at(bits_f, g.W, ra, ia)) continue;
                        if (!bit_at(bits_f, g.W, rb, ib)) continue;
                        const int la = label_f[(size_t)ra * g.nx + ia], lb = label_f[(size_t)rb * g.nx + ib];
                        if (la == lb) continue;
                        set_insert(table, mask, pair_key(f, la < lb ? la : lb, la < lb ? lb : la), overflow);
                    }
                }
            }
        }
    }
}

__global__ void k_compact_set(const unsigned long long* __restrict__ table, int cap,
                              unsigned long long* __restrict__ out, unsigned long long* count) {
    for (int base = blockIdx.x * blockDim.x; base < cap; base += gridDim.x * blockDim.x) {
        int s = base + threadIdx.x;
        unsigned long long key = s < cap ? table[s] : kEmptyKey;
        long long slot = warp_append(key != kEmptyKey, count);
        if (slot >= 0) out[slot] = key;
    }
}

cudaError_t tag_pairs_fields(const uint32_t* ncmap, const uint32_t* bits, const int* labels, const Dims& g, int w,
                             const LabelSlots& ls, unsigned long long* table, int cap, int* overflow,
                             cudaStream_t st) {
    if (ls.n <= 0) return cudaSuccess;
    if (ls.n > kLabelSlots) return cudaErrorInvalidValue;
    const long long words = (long long)g.rows * g.W;
    const int blocks = grid_for(words, 128, std::max(1, sm_count() * 32 / ls.n));
    k_pairs<<<dim3(blocks, ls.n), 128, 0, st>>>(ncmap, bits, labels, g, w, table, cap - 1, overflow, ls);
    return cudaGetLastError();
}

cudaError_t compact_pairs(const unsigned long long* table, int cap, unsigned long long* out,
                          unsigned long long* count, cudaStream_t st) {
    k_compact_set<<<grid_for(cap, 256), 256, 0, st>>>(table, cap, out, count);
    return cudaGetLastError();
}

}  // namespace vof
