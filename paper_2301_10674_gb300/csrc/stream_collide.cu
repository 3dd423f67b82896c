// Fused stream + boundary conditions + mass exchange + cumulant collision
// (Sections 2.1 and 2.2), in place with the AA pattern.
//
// Even step: each cell reads its own slots (q, x), writes (opp(q), x).
// Odd step: each cell reads (opp(q), x - c_q), writes (q, x + c_q).
// Every boundary condition is applied where a PDF is read: the value a cell
// needs for bounce-back or reconstruction is its own post-collision PDF
// f*_opp(q)(x), which sits in a slot no running cell touches (the slot of a
// solid/gas neighbour, or of the cell itself across a wall face). Interface
// cells read it from a side buffer instead, because the normal-based
// reconstruction also replaces PDFs pulled from fluid neighbours, whose slots
// are being rewritten.
//
// The work per step: the particle links from the solid side (they place the
// moving bounce-back values in the pull slots and gather the momentum
// exchange); the liquid cells (x-adjacent pairs per thread on packed FP32
// arithmetic; one cell per thread where nx is odd or the lattice needs
// 64-bit element indices); and the interface cells of the interface list.
#include "collide_pair.cuh"
#include "fslbm_dev.cuh"

namespace fsl {

// offsets of the x, y, z neighbours (-1, 0, +1) of a cell with the wall
// faces it touches as bits (x-, x+, y-, y+, z-, z+)
struct NbrOffsets {
    int ox[3], oy[3], oz[3];
    unsigned wall;
};
__device__ __forceinline__ NbrOffsets nbr_offsets(const Dev& s, int x, int y, int z) {
    const int sxy = s.nx * s.ny;
    NbrOffsets o;
    o.wall = 0;
    o.ox[0] = -1; o.ox[1] = 0; o.ox[2] = 1;
    o.oy[0] = -s.nx; o.oy[1] = 0; o.oy[2] = s.nx;
    o.oz[0] = -sxy; o.oz[1] = 0; o.oz[2] = sxy;
    if (x == 0) { if (s.per_x) o.ox[0] = s.nx - 1; else o.wall |= 1u; }
    if (x == s.nx - 1) { if (s.per_x) o.ox[2] = 1 - s.nx; else o.wall |= 2u; }
    if (y == 0) { if (s.per_y) o.oy[0] = (s.ny - 1) * s.nx; else o.wall |= 4u; }
    if (y == s.ny - 1) { if (s.per_y) o.oy[2] = (1 - s.ny) * s.nx; else o.wall |= 8u; }
    if (z == 0) { if (s.per_z) o.oz[0] = (s.nz - 1) * sxy; else o.wall |= 16u; }
    if (z == s.nz - 1) { if (s.per_z) o.oz[2] = (1 - s.nz) * sxy; else o.wall |= 32u; }
    return o;
}
// wall bits a direction d crosses from a cell
__host__ __device__ constexpr unsigned wall_bits(int dx, int dy, int dz) {
    return (dx == -1 ? 1u : 0u) | (dx == 1 ? 2u : 0u) | (dy == -1 ? 4u : 0u) | (dy == 1 ? 8u : 0u) |
           (dz == -1 ? 16u : 0u) | (dz == 1 ? 32u : 0u);
}

// All liquid cells. Every PDF is a plain pull: PDFs from fluid cells, and
// from solid cells the bounce-back values k_solid_links placed in the pull
// slots. Only wall faces need handling here, and they follow from the
// coordinates: an even step reads its own slots (a wall-bound PDF came back
// into (q, x) in the previous odd step), an odd step reads (q, x) across a
// wall face and writes (opp(q), x) toward one. Interior cells of an odd step
// use offsets that are the same for every thread. Blocks run over a
// 256-cell segment of a row (y, z), so the coordinates need no division per
// cell; the segment's liquid cells are compacted onto the first threads.
// Stored values move raw (times the storage scale); the collision folds the
// scale into its moments.
// resident blocks per SM asked of the compiler: 64 registers for FP32 storage,
// 48 for 16-bit storage (a few spilled words cost less than the lost warps)
template <typename S>
constexpr int liquid_min_blocks() { return sizeof(S) == 2 ? 5 : 4; }

template <typename S, int PAR>
__global__ void __launch_bounds__(256, liquid_min_blocks<S>()) k_liquid(Dev s) {
    __shared__ int xs[256];      // x of the liquid cells of this block's row segment, compacted
    __shared__ int wn[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    S* f = static_cast<S*>(s.f);
    const long long n = s.n;
    const int nrows = s.ny * s.nz;
    const int sxy = s.nx * s.ny;
    for (int row = blockIdx.y; row < nrows; row += gridDim.y) {
        // compaction: thread t collides the t-th liquid cell of the segment,
        // so only the last busy warp has idle lanes
        const int xt = blockIdx.x * blockDim.x + threadIdx.x;
        const bool liq = xt < s.nx && (s.flags[xt + s.nx * row] & TYPE_MASK) == T_LIQ;
        const unsigned m = __ballot_sync(0xffffffffu, liq);
        if (lane == 0) wn[warp] = __popc(m);
        __syncthreads();
        int off = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            off += w < warp ? wn[w] : 0;
            tot += wn[w];
        }
        if (liq) xs[off + __popc(m & ((1u << lane) - 1u))] = xt;
        __syncthreads();
        const int x = (int)threadIdx.x < tot ? xs[threadIdx.x] : -1;
        __syncthreads();             // xs and wn are rewritten by the next row
        if (x < 0) continue;
        const int cell = x + s.nx * row;
        const int y = row % s.ny, z = row / s.ny;
        const bool interior =
            PAR == 0 || (x > 0 && x < s.nx - 1 && y > 0 && y < s.ny - 1 && z > 0 && z < s.nz - 1);
        float v[27];
        if (interior && s.idx32) {
            const unsigned un = (unsigned)n;
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                const unsigned a = PAR == 0 ? (unsigned)q * un + (unsigned)cell
                                            : (unsigned)opp(q) * un +
                                                  (unsigned)(cell - (cx(q) + s.nx * cy(q) + sxy * cz(q)));
                v[q] = Store<S>::ld_raw(f + a);
            }
        } else if (interior) {
#pragma unroll
            for (int q = 0; q < 27; ++q)
                v[q] = Store<S>::ld_raw(PAR == 0 ? f + (long long)q * n + cell : f + cell + s.pull_off[q]);
        } else {
            const NbrOffsets o = nbr_offsets(s, x, y, z);
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                // source x - c_q beyond a wall face?
                const int src = cell + o.ox[1 - cx(q)] + o.oy[1 - cy(q)] + o.oz[1 - cz(q)];
                const long long a = (o.wall & wall_bits(-cx(q), -cy(q), -cz(q))) ? (long long)q * n + cell
                                                                                   : (long long)opp(q) * n + src;
                v[q] = Store<S>::ld_raw(f + a);
            }
        }
        if (Store<S>::HREF) {
            // deviations from w: each slot's reference added (the slot read is
            // the cell's own in an even step or across a wall face, else the
            // one at z - c_z)
            const NbrOffsets o = nbr_offsets(s, x, y, z);
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                const bool own = PAR == 0 || (o.wall & wall_bits(-cx(q), -cy(q), -cz(q)));
                v[q] += Store<S>::scale * wq(q) * s.href[own ? z : wrap_z(s, z - cz(q))];
            }
        }
        float rho, ux, uy, uz;
        collide_scaled(v, Store<S>::scale, s.omega, s.gx, s.gy, s.gz, rho, ux, uy, uz, s.galilean != 0);
        if (Store<S>::HREF) {
            const NbrOffsets o = nbr_offsets(s, x, y, z);
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                const bool own = PAR == 0 || (o.wall & wall_bits(cx(q), cy(q), cz(q)));
                v[q] -= Store<S>::scale * wq(q) * s.href[own ? z : wrap_z(s, z + cz(q))];
            }
        }
        if (interior && s.idx32) {
            const unsigned un = (unsigned)n;
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                const unsigned a = PAR == 0 ? (unsigned)opp(q) * un + (unsigned)cell
                                            : (unsigned)q * un +
                                                  (unsigned)(cell + cx(q) + s.nx * cy(q) + sxy * cz(q));
                Store<S>::st_raw(f + a, v[q]);
            }
        } else if (interior) {
#pragma unroll
            for (int q = 0; q < 27; ++q)
                Store<S>::st_raw(PAR == 0 ? f + (long long)opp(q) * n + cell : f + cell + s.push_off[q], v[q]);
        } else {
            const NbrOffsets o = nbr_offsets(s, x, y, z);
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                // target x + c_q beyond a wall face?
                const int dst = cell + o.ox[1 + cx(q)] + o.oy[1 + cy(q)] + o.oz[1 + cz(q)];
                const long long a = (o.wall & wall_bits(cx(q), cy(q), cz(q))) ? (long long)opp(q) * n + cell
                                                                               : (long long)q * n + dst;
                Store<S>::st_raw(f + a, v[q]);
            }
        }
    }
}

// The liquid cells as x-adjacent pairs (x even, x + 1), one pair per
// thread: the collision runs on packed FP32 pairs, a direction whose source
// or target keeps the pair's alignment (every direction in an even step,
// c_x = 0 in an odd one) moves both values with one aligned access, and the
// others with two accesses from one address. Blocks run over a 256-cell
// segment of a row; the segment's pairs that hold a liquid cell are
// compacted onto the first threads. A pair with one liquid cell collides
// both and stores only the liquid one (the other cell's pull slots are
// written by no thread of the sweep, so reading them races with nothing).
// Needs nx even and 32-bit element indices.
// Resident blocks per SM asked of the compiler, measured per parity: an
// even step (all accesses aligned pairs) runs fastest without spills (4
// blocks, up to 128 registers), an odd step with more warps (7 blocks for
// 16-bit storage, 5 for FP32).
template <typename S, int PAR>
constexpr int liquid_pair_min_blocks() { return PAR == 0 ? 4 : (sizeof(S) == 2 ? 7 : 5); }

// Stream and collide one pair (x even, x + 1) of row `row`; liq: bit 0 cell
// x liquid, bit 1 cell x + 1 liquid. `interior`: every neighbour of both
// cells inside the lattice without wrap (always true in an even step, which
// touches only a cell's own slots). In two halves, so that the bed kernel can
// replace the values pulled from particle cells in between: pair_load pulls
// the PDFs (v, with the references ref of the slots read and wt of the slots
// written), pair_finish collides and stores them.
template <typename S, int PAR>
__device__ __forceinline__ void pair_load(const Dev& s, const S* f, int x, int row, unsigned liq, bool interior,
                                          float2 (&v)[27], PairRef& ref, float (&wt)[3]) {
    const unsigned un = (unsigned)s.n;
    const int sxy = s.nx * s.ny;
    const int cell = x + s.nx * row;
    const int y = row % s.ny, z = row / s.ny;
    constexpr float SC = Store<S>::scale;
    // storage references (16-bit storage): interior pairs fold them into the
    // collision (even step: every slot at z; odd step: direction c_z read
    // from z - c_z, written to z + c_z); the others add and remove them value
    // by value and collide with zero references
#pragma unroll
    for (int k = 0; k < 3; ++k) ref.rd[k] = 0.f;
    // wt: reference of the slots written along c_z = -1, 0, +1
#pragma unroll
    for (int k = 0; k < 3; ++k) wt[k] = 0.f;
    if (interior) {
#pragma unroll
        for (int q = 0; q < 27; ++q) {
            const unsigned a = PAR == 0 ? (unsigned)q * un + (unsigned)cell
                                        : (unsigned)opp(q) * un +
                                              (unsigned)(cell - (cx(q) + s.nx * cy(q) + sxy * cz(q)));
            if (PAR == 0 || cx(q) == 0) v[q] = Pair<S>::ld2(f + a);
            else v[q] = make_float2(Store<S>::ld_raw(f + a), Store<S>::ld_raw(f + a + 1));
        }
        if (Store<S>::HREF) {
            const float h0 = s.href[z];
            if (PAR == 0) {
                ref.rd[0] = ref.rd[1] = ref.rd[2] = wt[0] = wt[1] = wt[2] = h0;
            } else {
                const float hm = s.href[z - 1], hp = s.href[z + 1];
                ref.rd[0] = hp; ref.rd[1] = h0; ref.rd[2] = hm;
                wt[0] = hm; wt[1] = h0; wt[2] = hp;
            }
        }
    } else {
        const NbrOffsets o0 = nbr_offsets(s, x, y, z), o1 = nbr_offsets(s, x + 1, y, z);
#pragma unroll
        for (int q = 0; q < 27; ++q) {
            // source x - c_q beyond a wall face: the cell's own slot (q, x)
            const unsigned wb = wall_bits(-cx(q), -cy(q), -cz(q));
            const int src0 = cell + o0.ox[1 - cx(q)] + o0.oy[1 - cy(q)] + o0.oz[1 - cz(q)];
            const int src1 = cell + 1 + o1.ox[1 - cx(q)] + o1.oy[1 - cy(q)] + o1.oz[1 - cz(q)];
            const long long a0 = (o0.wall & wb) ? (long long)q * s.n + cell : (long long)opp(q) * s.n + src0;
            const long long a1 =
                (o1.wall & wb) ? (long long)q * s.n + cell + 1 : (long long)opp(q) * s.n + src1;
            v[q] = make_float2((liq & 1u) ? Store<S>::ld_raw(f + a0) : 0.f,
                               (liq & 2u) ? Store<S>::ld_raw(f + a1) : 0.f);
            if (Store<S>::HREF) {
                const float hs = SC * wq(q) * s.href[wrap_z(s, z - cz(q))], ho = SC * wq(q) * s.href[z];
                v[q].x += (o0.wall & wb) ? ho : hs;
                v[q].y += (o1.wall & wb) ? ho : hs;
            }
        }
    }
}

template <typename S, int PAR>
__device__ __forceinline__ void pair_finish(const Dev& s, S* f, int x, int row, unsigned liq, bool interior,
                                            float2 (&v)[27], const PairRef& ref, const float (&wt)[3]) {
    const unsigned un = (unsigned)s.n;
    const int sxy = s.nx * s.ny;
    const int cell = x + s.nx * row;
    const int y = row % s.ny, z = row / s.ny;
    constexpr float SC = Store<S>::scale;
    collide_pair<Pair<S>::SCALE_LOG2, Store<S>::HREF>(v, s.omega, s.gx, s.gy, s.gz, ref);
    if (Store<S>::HREF && interior) {
        // each output loses the reference of the slot it is written to
#pragma unroll
        for (int q = 0; q < 27; ++q) v[q] = p_fma(p_set(-SC * wq(q)), p_set(wt[1 + cz(q)]), v[q]);
    }
    if (interior && liq == 3u) {
#pragma unroll
        for (int q = 0; q < 27; ++q) {
            const unsigned a = PAR == 0 ? (unsigned)opp(q) * un + (unsigned)cell
                                        : (unsigned)q * un +
                                              (unsigned)(cell + cx(q) + s.nx * cy(q) + sxy * cz(q));
            if (PAR == 0 || cx(q) == 0) {
                Pair<S>::st2(f + a, v[q]);
            } else {
                Store<S>::st_raw(f + a, v[q].x);
                Store<S>::st_raw(f + a + 1, v[q].y);
            }
        }
    } else if (interior) {
        // one liquid cell: liq is 1 (x) or 2 (x + 1)
        const unsigned k = liq >> 1;
#pragma unroll
        for (int q = 0; q < 27; ++q) {
            const unsigned a = PAR == 0 ? (unsigned)opp(q) * un + (unsigned)cell
                                        : (unsigned)q * un +
                                              (unsigned)(cell + cx(q) + s.nx * cy(q) + sxy * cz(q));
            Store<S>::st_raw(f + a + k, k ? v[q].y : v[q].x);
        }
    } else {
        const NbrOffsets o0 = nbr_offsets(s, x, y, z), o1 = nbr_offsets(s, x + 1, y, z);
#pragma unroll
        for (int q = 0; q < 27; ++q) {
            // target x + c_q beyond a wall face: the cell's own slot (opp(q), x)
            const unsigned wb = wall_bits(cx(q), cy(q), cz(q));
            const int dst0 = cell + o0.ox[1 + cx(q)] + o0.oy[1 + cy(q)] + o0.oz[1 + cz(q)];
            const int dst1 = cell + 1 + o1.ox[1 + cx(q)] + o1.oy[1 + cy(q)] + o1.oz[1 + cz(q)];
            float2 e = v[q];
            if (Store<S>::HREF) {
                const float ht = SC * wq(q) * s.href[wrap_z(s, z + cz(q))], ho = SC * wq(q) * s.href[z];
                e.x -= (o0.wall & wb) ? ho : ht;
                e.y -= (o1.wall & wb) ? ho : ht;
            }
            if (liq & 1u)
                Store<S>::st_raw(
                    f + ((o0.wall & wb) ? (long long)opp(q) * s.n + cell : (long long)q * s.n + dst0), e.x);
            if (liq & 2u)
                Store<S>::st_raw(
                    f + ((o1.wall & wb) ? (long long)opp(q) * s.n + cell + 1 : (long long)q * s.n + dst1),
                    e.y);
        }
    }
}

template <typename S, int PAR>
__device__ __forceinline__ void pair_update(const Dev& s, S* f, int x, int row, unsigned liq, bool interior) {
    float2 v[27];
    PairRef ref;
    float wt[3];
    pair_load<S, PAR>(s, f, x, row, liq, interior, v, ref, wt);
    pair_finish<S, PAR>(s, f, x, row, liq, interior, v, ref, wt);
}

// PART 1 keeps to the interior pairs of an odd step (all 26 neighbours of
// both cells inside the lattice, no wrap), so that the kernel of the bulk
// carries no boundary code; k_liquid_pair_edges takes the others. PART 0:
// every pair (even steps).
template <typename S, int PAR, int PART>
__global__ void __launch_bounds__(128, liquid_pair_min_blocks<S, PAR>()) k_liquid_pair(Dev s) {
    __shared__ int ps[128];      // (x << 2 | liquid bits) of the compacted pairs
    __shared__ int wn[4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    S* f = static_cast<S*>(s.f);
    const int nrows = s.ny * s.nz;
    for (int row = blockIdx.y; row < nrows; row += gridDim.y) {
        // the bed kernel takes the segments with particle links (the whole
        // block skips the row together)
        if (s.links_fused && s.segflag[row * s.nsegx + blockIdx.x]) continue;
        const int yr = row % s.ny, zr = row / s.ny;
        const bool face_row = yr == 0 || yr == s.ny - 1 || zr == 0 || zr == s.nz - 1;
        const int x0 = blockIdx.x * 256 + 2 * (int)threadIdx.x;
        unsigned lm = 0;
        if (x0 < s.nx) {
            const bool inner_pair = !face_row && x0 > 0 && x0 + 1 < s.nx - 1;
            if (PART == 0 || inner_pair) {
                const uchar2 fl = *reinterpret_cast<const uchar2*>(s.flags + x0 + (long long)s.nx * row);
                lm = ((fl.x & TYPE_MASK) == T_LIQ ? 1u : 0u) | ((fl.y & TYPE_MASK) == T_LIQ ? 2u : 0u);
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, lm != 0);
        if (lane == 0) wn[warp] = __popc(m);
        __syncthreads();
        int off = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            off += w < warp ? wn[w] : 0;
            tot += wn[w];
        }
        if (lm) ps[off + __popc(m & ((1u << lane) - 1u))] = (x0 << 2) | (int)lm;
        __syncthreads();
        const int e = (int)threadIdx.x < tot ? ps[threadIdx.x] : -1;
        __syncthreads();             // ps and wn are rewritten by the next row
        if (e < 0) continue;
        const int x = e >> 2;
        const bool interior =
            PAR == 0 || PART == 1 || (x > 0 && x + 1 < s.nx - 1 && !face_row);
        pair_update<S, PAR>(s, f, x, row, (unsigned)e & 3u, interior);
    }
}

// The pairs of an odd step that k_liquid_pair<S, 1, 1> leaves out, one per
// thread: every pair of the rows on the y and z faces, then the pairs at
// x = 0 and x = nx - 2 of the other rows (ny, nz >= 3 and nx >= 4, so that
// no pair is listed twice).
template <typename S>
__global__ void __launch_bounds__(128) k_liquid_pair_edges(Dev s) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int hp = s.nx / 2;                                   // pairs per row
    const long long nface = 2LL * s.nz + 2LL * (s.ny > 2 ? s.ny - 2 : 0);
    int y, z, x;
    if (t < nface * hp) {
        const int r = (int)(t / hp);
        x = 2 * (int)(t % hp);
        if (r < 2 * s.nz) { z = r >> 1; y = (r & 1) ? s.ny - 1 : 0; }
        else { const int k = r - 2 * s.nz; y = 1 + (k >> 1); z = (k & 1) ? s.nz - 1 : 0; }
    } else if (t < nface * hp + 2LL * (s.ny - 2) * (s.nz - 2)) {
        const long long k = t - nface * hp;
        x = (k & 1) ? s.nx - 2 : 0;
        const long long r = k >> 1;
        y = 1 + (int)(r % (s.ny - 2));
        z = 1 + (int)(r / (s.ny - 2));
    } else {
        return;
    }
    const int row = y + s.ny * z;
    if (s.links_fused && s.segflag[row * s.nsegx + x / BED_SEG]) return;   // a bed segment
    const uchar2 fl = *reinterpret_cast<const uchar2*>(s.flags + x + (long long)s.nx * row);
    const unsigned lm = ((fl.x & TYPE_MASK) == T_LIQ ? 1u : 0u) | ((fl.y & TYPE_MASK) == T_LIQ ? 2u : 0u);
    if (!lm) return;
    pair_update<S, 1>(s, static_cast<S*>(s.f), x, row, lm, false);
}

// ---------------------------------------------------------------- staged even step
// Even steps at 16-bit storage, tile by tile: a persistent CTA of SP_TILE/2
// threads streams the 27 direction slices [c0, c0 + SP_TILE) of each
// SP_TILE-cell x-tile that holds a liquid cell (and its flag bytes) into
// shared memory with bulk asynchronous copies (cp.async.bulk, completion
// counted on an mbarrier), STAGES tiles ahead, while its threads collide the
// tile in hand as x-adjacent pairs and write the results back with aligned
// pair stores. An even step reads and writes only a cell's own slots, so
// cells on the faces of the lattice need nothing else. Every copy starts and
// ends on a 16-byte boundary (nx is a multiple of SP_TILE). Every wait is
// bounded: one that gives up sets the timeout bit, the block leaves its loop
// on a block-wide vote, and the copies in flight are waited for before the
// block exits.
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: false (and the sticky timeout bit) if the phase has not
// completed after `limit` polls
__device__ __forceinline__ bool mbar_wait(const Dev& s, uint64_t* bar, unsigned parity, int limit) {
    for (int it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    set_error(s, ERR_TIMEOUT);
    return false;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// the x-tiles of SP_TILE cells that hold at least one liquid cell, in the
// order of their first cell within each block; SP_FULL marks a tile whose
// cells are all liquid
constexpr int SP_FULL = 1 << 30;
__global__ void k_sp_tiles(Dev s) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long ntile = s.n / SP_TILE;
    bool act = false;
    int val = (int)t;
    if (t < ntile) {
        const uint4* w = reinterpret_cast<const uint4*>(s.flags + t * SP_TILE);
        unsigned any = 0, other = 0;
#pragma unroll 4
        for (int k = 0; k < SP_TILE / 16; ++k) {
            const uint4 v = w[k];
            const unsigned wd[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                // a byte holds a liquid cell when its type bits are 01
                const unsigned lo = (wd[j] & 0x03030303u) ^ 0x01010101u;
                any |= (lo - 0x01010101u) & ~lo & 0x80808080u;
                other |= lo;
            }
        }
        // bed tiles (the same 256-cell x-ranges as the bed segments) are the
        // bed kernel's
        act = any != 0 && !(s.links_fused && s.segflag[t]);
        if (other == 0) val |= SP_FULL;
    }
    block_append(s, act, val, s.tiles, s.tile_count, (int)ntile);
}

template <typename S>
struct StagedPairLayout {
    static constexpr int STAGES = 2;
    static constexpr int ROW = SP_TILE;                          // elements per direction slice
    static constexpr int PDF_BYTES = 27 * ROW * (int)sizeof(S);
    static constexpr int STAGE_BYTES = PDF_BYTES + SP_TILE;      // + the tile's flag bytes
    static constexpr int SMEM = STAGES * STAGE_BYTES;
};

template <typename S>
__device__ __forceinline__ void staged_pair_issue(const Dev& s, unsigned char* stage, uint64_t* full, int tile) {
    using L = StagedPairLayout<S>;
    const S* f = static_cast<const S*>(s.f);
    const long long n = s.n;
    const long long c0 = (long long)(tile & ~SP_FULL) * SP_TILE;
    S* buf = reinterpret_cast<S*>(stage);
    mbar_expect_tx(full, (unsigned)L::STAGE_BYTES);
    bulk_load(stage + L::PDF_BYTES, s.flags + c0, SP_TILE, full);
#pragma unroll 1
    for (int q = 0; q < 27; ++q)
        bulk_load(buf + q * L::ROW, f + (long long)q * n + c0, SP_TILE * (unsigned)sizeof(S), full);
}

template <typename S>
__global__ void __launch_bounds__(SP_TILE / 2, 6) k_liquid_staged_pair(Dev s) {
    using L = StagedPairLayout<S>;
    constexpr int STAGES = L::STAGES;
    constexpr int NT = SP_TILE / 2;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[STAGES];
    __shared__ __align__(8) uint64_t empty[STAGES];
    __shared__ int stage_tile[STAGES];
    __shared__ int pos[NT];              // (pair << 2 | liquid bits) of the compacted pairs
    __shared__ int wn[NT / 32];
    const int ntiles = *s.tile_count;
    const int mine = ntiles > (int)blockIdx.x ? (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    if (mine == 0) return;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    auto issue = [&](int k, int i) {
        const int t = s.tiles[(int)blockIdx.x + i * (int)gridDim.x];
        stage_tile[k] = t;
        staged_pair_issue<S>(s, smem_raw + k * L::STAGE_BYTES, &full[k], t);
    };
    if (tid == 0) {
        for (int k = 0; k < STAGES; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], NT / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0)
        for (int k = 0; k < STAGES && k < mine; ++k) issue(k, k);
    S* f = static_cast<S*>(s.f);
    const unsigned un = (unsigned)s.n;
    // thread 0: the last tile index issued into each stage (-1: none), and
    // whether a refill gave up waiting for its stage to be released
    int last_issued[STAGES];
    bool refill_failed = false;
    for (int k = 0; k < STAGES; ++k) last_issued[k] = k < mine ? k : -1;
    for (int i = 0; i < mine; ++i) {
        const int st = i % STAGES;
        const unsigned ph = (unsigned)(i / STAGES) & 1u;
        const bool ok = mbar_wait(s, &full[st], ph, s.wait_limit);
        const unsigned char* stage = smem_raw + st * L::STAGE_BYTES;
        const S* buf = reinterpret_cast<const S*>(stage);
        const unsigned char* fl = stage + L::PDF_BYTES;
        // a bounded wait that gave up ends the loop for every thread at once;
        // the vote also keeps the next tile's compaction off pos and wn
        // until every thread has read them
        if (__syncthreads_or(!ok || refill_failed)) break;
        const int traw = stage_tile[st];
        int e = (tid << 2) | 3;
        if (!(traw & SP_FULL)) {
            // compaction: thread t collides the t-th pair of the tile that
            // holds a liquid cell
            const uchar2 b = *reinterpret_cast<const uchar2*>(fl + 2 * tid);
            const unsigned lm = ((b.x & TYPE_MASK) == T_LIQ ? 1u : 0u) | ((b.y & TYPE_MASK) == T_LIQ ? 2u : 0u);
            const unsigned m = __ballot_sync(0xffffffffu, lm != 0);
            if (lane == 0) wn[warp] = __popc(m);
            __syncthreads();
            int off = 0, tot = 0;
#pragma unroll
            for (int w = 0; w < NT / 32; ++w) {
                off += w < warp ? wn[w] : 0;
                tot += wn[w];
            }
            if (lm) pos[off + __popc(m & ((1u << lane) - 1u))] = (tid << 2) | (int)lm;
            __syncthreads();
            e = tid < tot ? pos[tid] : -1;
        }
        const int cell = (traw & ~SP_FULL) * SP_TILE + 2 * (e >> 2);
        if (e >= 0) {
            const int p = 2 * (e >> 2);
            const unsigned liq = (unsigned)e & 3u;
            float2 v[27];
#pragma unroll
            for (int q = 0; q < 27; ++q) v[q] = Pair<S>::ld2(buf + q * L::ROW + p);
            // an even step reads and writes the cells' own slots: one reference
            PairRef ref;
            const float h0 = s.href[(unsigned)cell / ((unsigned)s.nx * (unsigned)s.ny)];
#pragma unroll
            for (int k = 0; k < 3; ++k) ref.rd[k] = h0;
            collide_pair<Pair<S>::SCALE_LOG2, true>(v, s.omega, s.gx, s.gy, s.gz, ref);
            // outputs relative to w (1 + delta(z)) for the cells' own slots
#pragma unroll
            for (int q = 0; q < 27; ++q) v[q] = p_fma(p_set(-Store<S>::scale * wq(q)), p_set(h0), v[q]);
            if (liq == 3u) {
#pragma unroll
                for (int q = 0; q < 27; ++q) Pair<S>::st2(f + ((unsigned)opp(q) * un + (unsigned)cell), v[q]);
            } else {
                const unsigned k = liq >> 1;
#pragma unroll
                for (int q = 0; q < 27; ++q)
                    Store<S>::st_raw(f + ((unsigned)opp(q) * un + (unsigned)cell + k), k ? v[q].y : v[q].x);
            }
        }
        // release the stage, then refill it with the tile STAGES ahead
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
        if (tid == 0 && i + STAGES < mine) {
            if (!mbar_wait(s, &empty[st], ph, s.wait_limit)) {
                refill_failed = true;
            } else {
                issue(st, i + STAGES);
                last_issued[st] = i + STAGES;
            }
        }
    }
    // copies still in flight complete before the CTA leaves (with the default
    // limit whatever the stage waits were given: these copies were issued
    // and land in this CTA's shared memory)
    if (tid == 0)
        for (int k = 0; k < STAGES; ++k)
            if (last_issued[k] >= 0)
                mbar_wait(s, &full[k], (unsigned)(last_issued[k] / STAGES) & 1u, WAIT_LIMIT_DEFAULT);
}

// Warp segmented reduction of per-lane (key, F, T) for runs of equal keys,
// then one FP64 atomic per run and component.
__device__ __forceinline__ void flush_mem(const Dev& s, int key, const float (&F)[3], const float (&T)[3]) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    if (!__any_sync(full, key >= 0)) return;
    int kprev = __shfl_up_sync(full, key, 1);
    bool head = (lane == 0) || (kprev != key);
    unsigned heads = __ballot_sync(full, head);
    unsigned below = heads & ((2u << lane) - 1u);
    int start = 31 - __clz(below);
    float v[6] = {F[0], F[1], F[2], T[0], T[1], T[2]};
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float t = __shfl_up_sync(full, v[k], off);
            if (lane - off >= start) v[k] += t;
        }
    }
    int knext = __shfl_down_sync(full, key, 1);
    bool tail = (lane == 31) || (knext != key);
    if (tail && key >= 0) {
        atomicAdd(&s.Fh[3 * key + 0], (double)v[0]);
        atomicAdd(&s.Fh[3 * key + 1], (double)v[1]);
        atomicAdd(&s.Fh[3 * key + 2], (double)v[2]);
        atomicAdd(&s.Th[3 * key + 0], (double)v[3]);
        atomicAdd(&s.Th[3 * key + 1], (double)v[4]);
        atomicAdd(&s.Th[3 * key + 2], (double)v[5]);
    }
}

// one run's force and torque straight to the particle's FP64 sums
__device__ __forceinline__ void flush_direct(const Dev& s, int key, const float (&F)[3], const float (&T)[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        atomicAdd(&s.Fh[3 * key + c], (double)F[c]);
        atomicAdd(&s.Th[3 * key + c], (double)T[c]);
    }
}

// particle surface velocity at a link midpoint and the link force
// (Section 2.2): f_q = f*_opp + 6 w_q c_q.u_b, force on the particle
// -c_q (f*_opp + f_q) - u_b (f*_opp - f_q) with zero-centred PDFs; torque
// about the centre. The offset from the centre is formed from the integer
// part and the FP32 fraction of the centre, so it is exact to FP32 rounding
// at any lattice size.
__device__ __forceinline__ int wrap_int(int d, int L, int periodic) {
    if (periodic) {
        if (d > L / 2) d -= L;
        else if (d < -L / 2) d += L;
    }
    return d;
}

struct PData {
    int4 xi;
    float4 xf, u, w;
};
__device__ __forceinline__ PData particle_data(const Dev& s, int p) {
    PData d;
    d.xi = s.Xi[p];
    d.xf = s.Xfr[p];
    d.u = s.Uf[p];
    d.w = s.Wf[p];
    return d;
}

// Moving bounce-back and momentum exchange (Section 2.2), from the solid
// side: for every surface solid cell s (owner p) and every fluid neighbour
// x = s + c_q, the PDF x will pull from s in direction q is
// f_q(x) = f*_opp(q)(x) + 6 w_q c_q.u_b, u_b the particle velocity at the
// link midpoint. It is written into the slot x pulls in the coming sweep:
// (q, x) before an even step, (opp(q), s) before an odd one; f*_opp(q)(x)
// is read from (opp(q), s) or (q, x) respectively. The force on the
// particle is -c_q (f*_opp + f_q) - u_b (f*_opp - f_q) with zero-centred
// PDFs, the torque (x_b - X_p) x F, both summed over the cell's links in
// closed form (phase 3); one owner per thread, so a warp segmented reduction
// gathers them.
template <typename S, int PAR>
__global__ void __launch_bounds__(256, 3) k_solid_links(Dev s) {
    const int count = min(*s.sl_count, s.sl_cap);
    const int stride = gridDim.x * blockDim.x;
    float injected = 0.f;   // mass the moving bounce-back adds to liquid cells
    // the list entry of the next pass is loaded one pass ahead
    int next = blockIdx.x * blockDim.x + threadIdx.x < count ? s.sl[blockIdx.x * blockDim.x + threadIdx.x] : 0;
    for (int base = blockIdx.x * blockDim.x; base < count; base += stride) {
        const int i = base + threadIdx.x;
        const int cell = next;
        next = i + stride < count ? s.sl[i + stride] : 0;
        int key = -1;
        float F[3] = {0.f, 0.f, 0.f}, T[3] = {0.f, 0.f, 0.f};
        if (i < count) {
            int x, y, z;
            coords32(s, cell, x, y, z);
            const int p = s.owner[cell];
            S* f = static_cast<S*>(s.f);
            const long long n = s.n;
            const NbrOffsets o = nbr_offsets(s, x, y, z);
            // phase 1: which neighbours are fluid (wall faces excluded)
            unsigned fluidm = 0, liqm = 0;
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                if (q == 13 || (o.wall & wall_bits(cx(q), cy(q), cz(q)))) continue;
                const int xn = cell + o.ox[1 + cx(q)] + o.oy[1 + cy(q)] + o.oz[1 + cz(q)];
                const int tn = s.flags[xn] & TYPE_MASK;
                fluidm |= (tn == T_LIQ || tn == T_IFC) ? (1u << q) : 0u;
                liqm |= tn == T_LIQ ? (1u << q) : 0u;
            }
            if (p < 0 || p >= s.np) {
                if (fluidm) set_error(s, ERR_INVARIANT);
                fluidm = 0;
            } else {
                key = p;
            }
            // phase 2: the post-collision PDFs the fluid neighbours send here
            float fo[27];
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                const int xn = cell + o.ox[1 + cx(q)] + o.oy[1 + cy(q)] + o.oz[1 + cz(q)];
                const long long a = PAR == 0 ? (long long)opp(q) * n + cell : (long long)q * n + xn;
                fo[q] = ((fluidm >> q) & 1u) ? Store<S>::ld(f + a) : 0.f;
            }
            // phase 3: bounce-back values and momentum exchange. With u_s the
            // particle velocity at the solid cell's centre (offset d_s from
            // the particle centre), the link midpoint lies at d_s + c_q/2, so
            // u_b = u_s + W x c_q/2 and c_q.u_b = c_q.u_s. With
            // corr_q = 6 w_q c_q.u_s and t_q = 2 f*_opp + corr_q the link force
            // is -c_q t_q + u_b corr_q, and the sums over the cell's links are
            //   F = -sum c t + u_s sum corr + W x (sum c corr) / 2,
            //   T = d_s x F + [(sum c corr) x u_s + (W sum |c|^2 corr - M W) / 2] / 2,
            // M = sum corr c c^T: per link only sums with the signs of c_q.
            if (fluidm) {
                const PData P = particle_data(s, p);
                const float ddx = (float)wrap_int(x - P.xi.x, s.nx, s.per_x) + 0.5f - P.xf.x;
                const float ddy = (float)wrap_int(y - P.xi.y, s.ny, s.per_y) + 0.5f - P.xf.y;
                const float ddz = (float)wrap_int(z - P.xi.z, s.nz, s.per_z) + 0.5f - P.xf.z;
                const float usx = P.u.x + (P.w.y * ddz - P.w.z * ddy);
                const float usy = P.u.y + (P.w.z * ddx - P.w.x * ddz);
                const float usz = P.u.z + (P.w.x * ddy - P.w.y * ddx);
                // 16-bit storage: references of the solid cell's z and of the
                // neighbour's (an even step reads at the solid cell and writes
                // at the neighbour, an odd step the other way round)
                const float hz = Store<S>::HREF ? s.href[z] : 0.f;
                const int zm = wrap_z(s, z - 1), zp = wrap_z(s, z + 1);
                const float hm = Store<S>::HREF ? s.href[zm] : 0.f, hp = Store<S>::HREF ? s.href[zp] : 0.f;
                float Ax = 0.f, Ay = 0.f, Az = 0.f, B = 0.f, Cx = 0.f, Cy = 0.f, Cz = 0.f, D = 0.f;
                float Mxx = 0.f, Myy = 0.f, Mzz = 0.f, Mxy = 0.f, Mxz = 0.f, Myz = 0.f;
#pragma unroll
                for (int q = 0; q < 27; ++q) {
                    if (!((fluidm >> q) & 1u)) continue;
                    const float hn = cz(q) == 0 ? hz : (cz(q) < 0 ? hm : hp);
                    if (Store<S>::HREF) fo[q] += wq(q) * (PAR == 0 ? hz : hn);
                    const int xn = cell + o.ox[1 + cx(q)] + o.oy[1 + cy(q)] + o.oz[1 + cz(q)];
                    // c_q.u_s with the signs of c_q
                    float cu = 0.f;
                    if (cx(q)) cu = cx(q) > 0 ? cu + usx : cu - usx;
                    if (cy(q)) cu = cy(q) > 0 ? cu + usy : cu - usy;
                    if (cz(q)) cu = cz(q) > 0 ? cu + usz : cu - usz;
                    const float corr = (6.f * wq(q)) * cu;
                    const float val = fo[q] + corr;
                    if ((liqm >> q) & 1u) injected += corr;
                    const long long dst = PAR == 0 ? (long long)q * n + xn : (long long)opp(q) * n + cell;
                    Store<S>::st(f + dst, Store<S>::HREF ? val - wq(q) * (PAR == 0 ? hn : hz) : val);
                    const float t = fmaf(2.f, fo[q], corr);
                    if (cx(q)) { Ax = cx(q) > 0 ? Ax + t : Ax - t; Cx = cx(q) > 0 ? Cx + corr : Cx - corr; Mxx += corr; }
                    if (cy(q)) { Ay = cy(q) > 0 ? Ay + t : Ay - t; Cy = cy(q) > 0 ? Cy + corr : Cy - corr; Myy += corr; }
                    if (cz(q)) { Az = cz(q) > 0 ? Az + t : Az - t; Cz = cz(q) > 0 ? Cz + corr : Cz - corr; Mzz += corr; }
                    if (cx(q) && cy(q)) Mxy = cx(q) * cy(q) > 0 ? Mxy + corr : Mxy - corr;
                    if (cx(q) && cz(q)) Mxz = cx(q) * cz(q) > 0 ? Mxz + corr : Mxz - corr;
                    if (cy(q) && cz(q)) Myz = cy(q) * cz(q) > 0 ? Myz + corr : Myz - corr;
                    B += corr;
                    D += (float)nnz(q) * corr;
                }
                const float hx = 0.5f * (P.w.y * Cz - P.w.z * Cy);
                const float hy = 0.5f * (P.w.z * Cx - P.w.x * Cz);
                const float hzz = 0.5f * (P.w.x * Cy - P.w.y * Cx);
                F[0] = fmaf(usx, B, hx) - Ax;
                F[1] = fmaf(usy, B, hy) - Ay;
                F[2] = fmaf(usz, B, hzz) - Az;
                // M W
                const float mwx = Mxx * P.w.x + Mxy * P.w.y + Mxz * P.w.z;
                const float mwy = Mxy * P.w.x + Myy * P.w.y + Myz * P.w.z;
                const float mwz = Mxz * P.w.x + Myz * P.w.y + Mzz * P.w.z;
                const float gx = (Cy * usz - Cz * usy) + 0.5f * (P.w.x * D - mwx);
                const float gy = (Cz * usx - Cx * usz) + 0.5f * (P.w.y * D - mwy);
                const float gz = (Cx * usy - Cy * usx) + 0.5f * (P.w.z * D - mwz);
                T[0] = (ddy * F[2] - ddz * F[1]) + 0.5f * gx;
                T[1] = (ddz * F[0] - ddx * F[2]) + 0.5f * gy;
                T[2] = (ddx * F[1] - ddy * F[0]) + 0.5f * gz;
            }
        }
        flush_mem(s, key, F, T);
    }
    // R-12a: the net injection leaves the pool (one FP64 atomic per block)
    if (s.link_corr) {
        __shared__ float red[8];
        for (int off = 16; off > 0; off >>= 1) injected += __shfl_xor_sync(0xffffffffu, injected, off);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = injected;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            if (t != 0.f) atomicAdd(s.pool, -(double)t);
        }
    }
}

// ---------------------------------------------------------------- bed segments
// Particle links from the fluid side (Section 2.2). A liquid cell x pulls f_q
// from a particle cell s = x - c_q as the moving bounce-back value
// f_q(x) = f*_opp(q)(x) + 6 w_q c_q.u_b, u_b the particle's surface velocity
// at the link midpoint x - c_q/2. The cell's own post-collision PDF
// f*_opp(q)(x) sits in a slot no running cell touches: (opp(q), s) before an
// even step (the odd step before pushed it there), (q, x) before an odd one.
// The force on the particle is -c_q (f*_opp + f_q) - u_b (f*_opp - f_q) with
// zero-centred PDFs, the torque (x_b - X_p) x F. These are the values and
// sums of the pass over the solid cells (k_solid_links), taken where the
// liquid cell is updated, so that the bed's PDFs cross HBM once per step.
//
// k_liquid_pair_bed updates every liquid pair of the bed segments listed by
// the classification (the bulk kernels skip them), a warp per 256-cell
// segment and no block-wide barrier. The warp stages the solid bit words of
// the 3x3 rows around its segment, compacts the segment's liquid pairs
// (interior pairs first, then those on the faces of the lattice), and takes
// them 32 at a time. Each pair reads its solid-neighbour masks from the
// words; the warp spreads the round's links evenly over its lanes (a
// contiguous run of links per lane, in the order pair, cell, direction),
// which compute the bounce-back values into shared memory and sum the
// momentum exchange per run of equal owner; the runs ending the lanes' shares
// merge across the warp (a segmented scan) into one FP64 atomic per run and
// component. The pair then pulls its PDFs as in the bulk kernels, takes the
// link values in place of those pulled from particle cells, collides and
// stores.
constexpr int BED_LINKS = 50;   // links of a pair at most (25 per liquid cell of a liquid pair)
static_assert(BED_SEG == 256 && SP_TILE == BED_SEG, "bed segments are the 256-cell blocks and tiles");

struct BedWarp {
    unsigned sw[9][10];              // solid words of rows (y + dy, z + dz), r = dy + 1 + 3 (dz + 1); halo words 0, 9
    int pairs[BED_SEG / 2];          // the segment's liquid pairs (x << 2 | liquid bits), interior ones first
    int lbase[33];                   // first link of each lane's pair in the round, and the round's total
    unsigned lm[2][32];              // solid masks of each lane's two cells
    int lx[32];                      // x of each lane's pair, bit 30 set for an interior pair
    float sval[32 * BED_LINKS];      // the round's link values, in link order
};

// The links of the round, lane `lane`'s share: links [lane C, lane C + C)
// of `total`, C = ceil(total / 32), four at a time (their owner and PDF loads
// issued together). Every lane of the warp calls it.
template <typename S, int PAR>
__device__ __forceinline__ void bed_links(BedWarp& sh, const Dev& s, const S* f, int lane, int row, int y, int z,
                                          int total, float& injected) {
    const int C = (total + 31) >> 5;
    const int t0 = min(lane * C, total), t1 = min(t0 + C, total);
    const unsigned un = (unsigned)s.n;
    int key = -1;
    float F[3] = {0.f, 0.f, 0.f}, T[3] = {0.f, 0.f, 0.f};
    PData P;
    P.xi = make_int4(0, 0, 0, 0);
    P.xf = P.u = P.w = make_float4(0.f, 0.f, 0.f, 0.f);
    if (t0 < t1) {
        int l = 0;
        while (sh.lbase[l + 1] <= t0) ++l;
        unsigned r0 = sh.lm[0][l], r1 = sh.lm[1][l];
        for (int r = t0 - sh.lbase[l]; r > 0; --r) {
            if (r0) r0 &= r0 - 1u;
            else r1 &= r1 - 1u;
        }
        for (int tb = t0; tb < t1; tb += 4) {
            int qq[4], xq[4], own[4];
            float fo[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                own[u] = -2;   // no link (beyond the share)
                qq[u] = 0;
                xq[u] = 0;
                fo[u] = 0.f;
                if (tb + u < t1) {
                    while (!(r0 | r1) && l < 31) {   // lanes without links hold none
                        ++l;
                        r0 = sh.lm[0][l];
                        r1 = sh.lm[1][l];
                    }
                    int q, kc;
                    if (r0) { q = __ffs(r0) - 1; r0 &= r0 - 1u; kc = 0; }
                    else if (r1) { q = __ffs(r1) - 1; r1 &= r1 - 1u; kc = 1; }
                    else { q = -1; kc = 0; }   // (the counts and masks disagree: cannot happen)
                    own[u] = -1;
                    if (q >= 0) {
                        const int lx = sh.lx[l];
                        const int xl = (lx & 0x3fffffff) + kc;
                        qq[u] = q;
                        xq[u] = xl | (lx & (1 << 30));
                        const int qx = q % 3 - 1, qy = (q / 3) % 3 - 1, qz = q / 9 - 1;
                        // the source x - c_q: inside the lattice (the masks
                        // hold no source beyond a wall face)
                        const int sx = shift(xl, -qx, s.nx, s.per_x), sy = shift(y, -qy, s.ny, s.per_y),
                                  sz = shift(z, -qz, s.nz, s.per_z);
                        if (sx >= 0 && sy >= 0 && sz >= 0) {
                            const int src = sx + s.nx * (sy + s.ny * sz);
                            own[u] = s.owner[src];
                            const unsigned a = PAR == 0 ? (unsigned)(26 - q) * un + (unsigned)src
                                                        : (unsigned)q * un + (unsigned)(xl + s.nx * row);
                            fo[u] = Store<S>::ld(f + a);
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (own[u] == -2) continue;
                const int t = tb + u;
                const int p = own[u];
                if (p < 0 || p >= s.np) {
                    set_error(s, ERR_INVARIANT);
                    sh.sval[t] = 0.f;
                    continue;
                }
                if (p != key) {
                    if (key >= 0) flush_direct(s, key, F, T);
                    key = p;
#pragma unroll
                    for (int c = 0; c < 3; ++c) F[c] = T[c] = 0.f;
                    P = particle_data(s, p);
                }
                const int q = qq[u];
                const int xl = xq[u] & 0x3fffffff;
                const bool interior = (xq[u] >> 30) & 1;
                const int qx = q % 3 - 1, qy = (q / 3) % 3 - 1, qz = q / 9 - 1;
                const int nzc = (qx != 0) + (qy != 0) + (qz != 0);
                const float w = nzc == 1 ? 2.f / 27.f : (nzc == 2 ? 1.f / 54.f : 1.f / 216.f);
                float fov = fo[u];
                if (Store<S>::HREF) fov += w * s.href[PAR == 0 ? wrap_z(s, z - qz) : z];
                const float dx = (float)wrap_int(xl - P.xi.x, s.nx, s.per_x) + 0.5f - P.xf.x - 0.5f * (float)qx;
                const float dy = (float)wrap_int(y - P.xi.y, s.ny, s.per_y) + 0.5f - P.xf.y - 0.5f * (float)qy;
                const float dz = (float)wrap_int(z - P.xi.z, s.nz, s.per_z) + 0.5f - P.xf.z - 0.5f * (float)qz;
                const float ubx = P.u.x + (P.w.y * dz - P.w.z * dy);
                const float uby = P.u.y + (P.w.z * dx - P.w.x * dz);
                const float ubz = P.u.z + (P.w.x * dy - P.w.y * dx);
                const float cu = (float)qx * ubx + (float)qy * uby + (float)qz * ubz;
                const float corr = 6.f * w * cu;
                const float val = fov + corr;
                injected += corr;
                // in the convention of the pair's pull: scaled, and relative
                // to the reference the collision assumes for the slot
                // (interior pairs: that of z in an even step, of z - c_z in
                // an odd one)
                float rexp = 0.f;
                if (Store<S>::HREF && interior) rexp = s.href[PAR == 0 ? z : z - qz];
                sh.sval[t] = Store<S>::scale * (val - w * rexp);
                const float sum = fov + val;
                const float Fx = -(float)qx * sum + ubx * corr;
                const float Fy = -(float)qy * sum + uby * corr;
                const float Fz = -(float)qz * sum + ubz * corr;
                F[0] += Fx; F[1] += Fy; F[2] += Fz;
                T[0] += dy * Fz - dz * Fy;
                T[1] += dz * Fx - dx * Fz;
                T[2] += dx * Fy - dy * Fx;
            }
        }
    }
    // the lanes' last runs, merged where adjacent lanes share the owner
    flush_mem(s, key, F, T);
}

// resident blocks per SM asked of the compiler: 6 for the even step (no
// spills), 5 for the odd one, whose pairs on the faces of the lattice take
// the boundary code
template <int PAR>
constexpr int bed_min_blocks() { return PAR == 0 ? 6 : 5; }

template <typename S, int PAR>
__global__ void __launch_bounds__(128, bed_min_blocks<PAR>()) k_liquid_pair_bed(Dev s) {
    __shared__ BedWarp shw[4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    BedWarp& sh = shw[warp];
    const unsigned full = 0xffffffffu;
    S* f = static_cast<S*>(s.f);
    const int count = min(*s.bseg_count, s.nsegx * s.ny * s.nz);
    const int nxw = s.nx >> 5;
    float injected = 0.f;
    for (int i = blockIdx.x * 4 + warp; i < count; i += gridDim.x * 4) {
        const int seg = s.bseg[i];
        const int row = seg / s.nsegx, xs = seg - row * s.nsegx;
        const int y = row % s.ny, z = row / s.ny;
        const bool face_row = y == 0 || y == s.ny - 1 || z == 0 || z == s.nz - 1;
        for (int k = lane; k < 90; k += 32) {
            const int r = k / 10, j = k - 10 * r;
            const int yy = shift(y, r % 3 - 1, s.ny, s.per_y), zz = shift(z, r / 3 - 1, s.nz, s.per_z);
            int xw = xs * (BED_SEG / 32) + j - 1;
            if (xw < 0) xw = s.per_x ? nxw - 1 : -1;
            else if (xw == nxw) xw = s.per_x ? 0 : -1;
            else if (xw > nxw) xw = -1;
            sh.sw[r][j] = (yy >= 0 && zz >= 0 && xw >= 0) ? s.sbits[((long long)zz * s.ny + yy) * nxw + xw] : 0u;
        }
        // the segment's liquid pairs: lane l looks at cells xb + 8l .. + 7
        // (pairs 4l .. 4l + 3; nx is a multiple of 32, so a segment holds
        // whole groups of eight)
        const int xb = xs * BED_SEG;
        const int xg = xb + 8 * lane;
        unsigned codes = 0;   // 4 bits per pair: liquid bits, and bit 2 for an interior pair
        if (xg < s.nx) {
            const uint2 fl = *reinterpret_cast<const uint2*>(s.flags + xg + (long long)s.nx * row);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const unsigned b = ((k < 2 ? fl.x : fl.y) >> (16 * (k & 1))) & 0xffffu;
                const unsigned lq = ((b & TYPE_MASK) == T_LIQ ? 1u : 0u) | (((b >> 8) & TYPE_MASK) == T_LIQ ? 2u : 0u);
                const int x = xg + 2 * k;
                const bool in = PAR == 0 || (x > 0 && x + 1 < s.nx - 1 && !face_row);
                codes |= (lq | (lq && in ? 4u : 0u)) << (4 * k);
            }
        }
        int ni = 0, nb = 0;   // interior and face pairs of this lane
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned c = (codes >> (4 * k)) & 0xFu;
            ni += (c & 4u) ? 1 : 0;
            nb += ((c & 3u) && !(c & 4u)) ? 1 : 0;
        }
        int ii = ni, ib = nb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int a = __shfl_up_sync(full, ii, o), b = __shfl_up_sync(full, ib, o);
            if (lane >= o) { ii += a; ib += b; }
        }
        const int n_int = __shfl_sync(full, ii, 31), n_all = n_int + __shfl_sync(full, ib, 31);
        {
            int pi = ii - ni, pb = n_int + ib - nb;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const unsigned c = (codes >> (4 * k)) & 0xFu;
                const int v = ((xg + 2 * k) << 2) | (int)(c & 3u);
                if (c & 4u) sh.pairs[pi++] = v;
                else if (c & 3u) sh.pairs[pb++] = v;
            }
        }
        __syncwarp();
        // rounds of 32 pairs: the interior ones, then those on the faces
        const int nr_int = (n_int + 31) >> 5, nr_all = nr_int + ((n_all - n_int + 31) >> 5);
        for (int rnd = 0; rnd < nr_all; ++rnd) {
            const bool in_phase = rnd < nr_int;
            const int lo = in_phase ? 32 * rnd : n_int + 32 * (rnd - nr_int);
            const int e = lo + lane < (in_phase ? n_int : n_all) ? sh.pairs[lo + lane] : -1;
            const bool act = e >= 0;
            const bool interior = PAR == 0 || in_phase;   // (every pair of an even step)
            const int x = act ? e >> 2 : 0;
            const unsigned liq = act ? (unsigned)e & 3u : 0u;
            // solid masks: bit q where the source x - c_q (x + 1 - c_q) of
            // the pair's liquid cell x (x + 1) is a particle cell
            unsigned qm0 = 0u, qm1 = 0u;
            if (act) {
                const int k = x - xb;   // even
                const int jw = 1 + (k >> 5), kb = k & 31;
                unsigned n0 = 0u, n1 = 0u;
#pragma unroll
                for (int r = 0; r < 9; ++r) {
                    // bit 1 + j: cell (x & ~31) + j of row r, j = -1 .. 32
                    const unsigned long long v64 = ((unsigned long long)sh.sw[r][jw] << 1) |
                                                   (sh.sw[r][jw - 1] >> 31) |
                                                   ((unsigned long long)(sh.sw[r][jw + 1] & 1u) << 33);
                    const unsigned b4 = (unsigned)(v64 >> kb) & 0xFu;   // cells x - 1 .. x + 2
                    n0 |= (b4 & 7u) << (3 * r);
                    n1 |= ((b4 >> 1) & 7u) << (3 * r);
                }
                // neighbour (dx, dy, dz) has index (dx+1) + 3(dy+1) + 9(dz+1),
                // which is 26 - q for the source of direction q
                qm0 = (liq & 1u) ? __brev(n0) >> 5 : 0u;
                qm1 = (liq & 2u) ? __brev(n1) >> 5 : 0u;
            }
            const int cnt = __popc(qm0) + __popc(qm1);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(full, incl, o);
                if (lane >= o) incl += t;
            }
            const int total = __shfl_sync(full, incl, 31);
            if (total) {
                sh.lbase[lane] = incl - cnt;
                if (lane == 31) sh.lbase[32] = total;
                sh.lm[0][lane] = qm0;
                sh.lm[1][lane] = qm1;
                sh.lx[lane] = x | (interior ? 1 << 30 : 0);
                __syncwarp();
                bed_links<S, PAR>(sh, s, f, lane, row, y, z, total, injected);
                __syncwarp();
            }
            if (act) {
                float2 v[27];
                PairRef ref;
                float wt[3];
                pair_load<S, PAR>(s, f, x, row, liq, interior, v, ref, wt);
                if (cnt) {
                    int pos = incl - cnt;
#pragma unroll
                    for (int q = 0; q < 27; ++q)
                        if ((qm0 >> q) & 1u) v[q].x = sh.sval[pos++];
#pragma unroll
                    for (int q = 0; q < 27; ++q)
                        if ((qm1 >> q) & 1u) v[q].y = sh.sval[pos++];
                }
                pair_finish<S, PAR>(s, f, x, row, liq, interior, v, ref, wt);
            }
            __syncwarp();   // lbase, lm, lx, sval free for the next round
        }
        __syncwarp();       // sw and pairs free for the next segment
    }
    // R-12a: the net injection into liquid cells leaves the pool (one FP64
    // atomic per warp)
    if (s.link_corr) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) injected += __shfl_xor_sync(full, injected, o);
        if (lane == 0 && injected != 0.f) atomicAdd(s.pool, -(double)injected);
    }
}

// Interface cells, from the interface list: gas-pressure reconstruction
// (Section 2.1), mass exchange, particle links, collision; the cell's own
// post-collision PDFs come from and go to the side buffer. Four blocks per
// SM (128 registers, a few dozen bytes of spills) rather than the two that
// the compiler's 250 registers leave: the kernel waits on dependent gathers.
template <typename S, int PAR>
__global__ void __launch_bounds__(128, 4) k_interface(Dev s) {
    const int count = min(*s.wl_count, s.wl_cap);
    const int stride = gridDim.x * blockDim.x;
    for (int base = blockIdx.x * blockDim.x; base < count; base += stride) {
        const int i = base + threadIdx.x;
        const bool work = i < count;
        // momentum exchange of the fluid-side particle links
        int lkey = -1;
        float LF[3] = {0.f, 0.f, 0.f}, LT[3] = {0.f, 0.f, 0.f};
        if (work) {
            const long long cell = s.wl[i];
            int x, y, z;
            coords32(s, (int)cell, x, y, z);
            S* f = static_cast<S*>(s.f);
            S* fs = static_cast<S*>(s.fs);
            const long long n = s.n;
            const int xs[3] = {shift(x, -1, s.nx, s.per_x), x, shift(x, 1, s.nx, s.per_x)};
            const int ys[3] = {shift(y, -1, s.ny, s.per_y), y, shift(y, 1, s.ny, s.per_y)};
            const int zs[3] = {shift(z, -1, s.nz, s.per_z), z, shift(z, 1, s.nz, s.per_z)};
            unsigned wallm = 0, solidm = 0, gasm = 0, liqm = 0;
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                const int sx = xs[1 - cx(q)], sy = ys[1 - cy(q)], sz = zs[1 - cz(q)];
                if (sx < 0 || sy < 0 || sz < 0) {
                    wallm |= 1u << q;
                } else {
                    const int ts = s.flags[sx + (long long)s.nx * (sy + (long long)s.ny * sz)] & TYPE_MASK;
                    if (ts == T_SOL) solidm |= 1u << q;
                    else if (ts == T_GAS) gasm |= 1u << q;
                    else if (ts == T_LIQ) liqm |= 1u << q;
                }
            }
            const float phix = s.phi[cell];
            const float mx = s.mass[cell];
            const float4 nn = s.nrm[cell];
            // 16-bit storage: references of the slots (the cell's own z, the
            // pull source's z - c_z in an odd step, the target's z + c_z); h3[k]
            // that of z + k - 1 (the cell's own beyond a wall face, never used)
            const float hz = Store<S>::HREF ? s.href[z] : 0.f;
            float h3[3] = {hz, hz, hz};
            if (Store<S>::HREF && PAR == 1) {
                if (zs[0] >= 0) h3[0] = s.href[zs[0]];
                if (zs[2] >= 0) h3[2] = s.href[zs[2]];
            }
            float fo[27];
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                fo[q] = Store<S>::ld(fs + (long long)q * n + cell);
                if (Store<S>::HREF) fo[q] += wq(q) * hz;
            }
            float v[27];
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                const int sx = xs[1 - cx(q)], sy = ys[1 - cy(q)], sz = zs[1 - cz(q)];
                const bool pull = !(((wallm | gasm) >> q) & 1u);   // fluid or solid source
                const long long src = pull ? sx + (long long)s.nx * (sy + (long long)s.ny * sz) : cell;
                const long long a = PAR == 0 ? (long long)q * n + cell : (long long)opp(q) * n + src;
                v[q] = pull ? Store<S>::ld(f + a) : 0.f;
                if (Store<S>::HREF && pull) v[q] += wq(q) * (PAR == 0 ? hz : h3[1 - cz(q)]);
            }
            // own collision velocity from the post-collision PDFs
            float d = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                d += fo[q];
                jx += cx(q) * fo[q];
                jy += cy(q) * fo[q];
                jz += cz(q) * fo[q];
            }
            const float rr = 1.f + d;
            const float urx = (jx - 0.5f * rr * s.gx) / rr;
            const float ury = (jy - 0.5f * rr * s.gy) / rr;
            const float urz = (jz - 0.5f * rr * s.gz) / rr;
            const float uur = urx * urx + ury * ury + urz * urz;
            // gas pressure plus the Laplace pressure 2 sigma kappa (Section 2.1),
            // kappa the curvature that came with the cell's normal (0 where
            // the finite-difference normal was taken)
            const float rhoG = s.rho_gas + 6.f * s.sigma * nn.w;
            float dm = 0.f;
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                const float fob = fo[opp(q)];
                if ((wallm >> q) & 1u) {
                    v[q] = fob;
                    continue;
                }
                const int sx = xs[1 - cx(q)], sy = ys[1 - cy(q)], sz = zs[1 - cz(q)];
                const long long src = sx + (long long)s.nx * (sy + (long long)s.ny * sz);
                // solid source: the pulled value is the bounce-back value,
                // placed by the link pass, or formed here from the cell's own
                // f*_opp(q) (its side-buffer copy) with the momentum exchange
                // summed per run of equal owner
                if ((solidm >> q) & 1u) {
                    if (s.links_fused) {
                        const int p = s.owner[src];
                        if (p < 0 || p >= s.np) {
                            set_error(s, ERR_INVARIANT);
                            continue;
                        }
                        if (p != lkey) {
                            if (lkey >= 0) flush_direct(s, lkey, LF, LT);
                            lkey = p;
#pragma unroll
                            for (int c = 0; c < 3; ++c) LF[c] = LT[c] = 0.f;
                        }
                        const PData P = particle_data(s, p);
                        const float dx = (float)wrap_int(x - P.xi.x, s.nx, s.per_x) + 0.5f - P.xf.x - 0.5f * cx(q);
                        const float dy = (float)wrap_int(y - P.xi.y, s.ny, s.per_y) + 0.5f - P.xf.y - 0.5f * cy(q);
                        const float dz = (float)wrap_int(z - P.xi.z, s.nz, s.per_z) + 0.5f - P.xf.z - 0.5f * cz(q);
                        const float ubx = P.u.x + (P.w.y * dz - P.w.z * dy);
                        const float uby = P.u.y + (P.w.z * dx - P.w.x * dz);
                        const float ubz = P.u.z + (P.w.x * dy - P.w.y * dx);
                        const float corr = 6.f * wq(q) * (cx(q) * ubx + cy(q) * uby + cz(q) * ubz);
                        v[q] = fob + corr;
                        const float sum = fob + v[q];
                        const float Fx = -cx(q) * sum + ubx * corr;
                        const float Fy = -cy(q) * sum + uby * corr;
                        const float Fz = -cz(q) * sum + ubz * corr;
                        LF[0] += Fx; LF[1] += Fy; LF[2] += Fz;
                        LT[0] += dy * Fz - dz * Fy;
                        LT[1] += dz * Fx - dx * Fz;
                        LT[2] += dx * Fy - dy * Fx;
                    }
                    continue;
                }
                const bool gas = (gasm >> q) & 1u;
                if (!gas) {
                    // fluid source: mass exchange with the pulled post-collision PDF
                    const bool liq = (liqm >> q) & 1u;
                    const float sc = liq ? 1.f : 0.5f * (phix + s.phi[src]);
                    dm += sc * (v[q] - fob);
                }
                bool rebuild = gas;
                if (!rebuild && s.recon_normal) rebuild = (nn.x * cx(q) + nn.y * cy(q) + nn.z * cz(q)) < -s.eps_normal;
                if (rebuild) {
                    const float cu = cx(q) * urx + cy(q) * ury + cz(q) * urz;
                    v[q] = wq(q) * (2.f * (rhoG - 1.f) + rhoG * (9.f * cu * cu - 3.f * uur)) - fob;
                }
            }
            float rho, ux, uy, uz;
            collide_scaled(v, 1.f, s.omega, s.gx, s.gy, s.gz, rho, ux, uy, uz, s.galilean != 0);
            if (PAR == 0) {
#pragma unroll
                for (int q = 0; q < 27; ++q)
                    Store<S>::st(f + (long long)opp(q) * n + cell, Store<S>::HREF ? v[q] - wq(q) * hz : v[q]);
            } else {
#pragma unroll
                for (int q = 0; q < 27; ++q) {
                    const int tx = xs[1 + cx(q)], ty = ys[1 + cy(q)], tz = zs[1 + cz(q)];
                    const bool out = tx < 0 || ty < 0 || tz < 0;
                    const long long a = out ? (long long)opp(q) * n + cell
                                            : (long long)q * n + tx + (long long)s.nx * (ty + (long long)s.ny * tz);
                    Store<S>::st(f + a, Store<S>::HREF ? v[q] - wq(q) * (out ? hz : h3[1 + cz(q)]) : v[q]);
                }
            }
#pragma unroll
            for (int q = 0; q < 27; ++q)
                Store<S>::st(fs + (long long)q * n + cell, Store<S>::HREF ? v[q] - wq(q) * hz : v[q]);
            // phi = m / rho is refreshed after the sweep: neighbours read the
            // old phi in their mass exchange
            s.mass[cell] = mx + dm;
            s.ru[cell] = make_float4(rho, ux, uy, uz);
        }
        flush_mem(s, lkey, LF, LT);
    }
}

// the pair collision carries no Galilean correction: with it every liquid
// cell runs in the one-cell kernel
static bool use_pairs(const Dev& s) { return s.idx32 && (s.nx % 2) == 0 && !s.galilean; }
// odd steps at 16-bit storage: interior pairs and the boundary pairs in two
// launches (at FP32 the odd step is bound by HBM, and one launch is faster)
static bool use_split(const Dev& s) {
    return use_pairs(s) && s.storage != FSLBM_STORE_FP32 && s.nx >= 4 && s.ny >= 3 && s.nz >= 3;
}
// the staged even step: 16-bit storage, nx a multiple of the tile
static bool use_staged_pairs(const Dev& s) {
    return s.idx32 && s.storage != FSLBM_STORE_FP32 && (s.nx % SP_TILE) == 0 && !s.galilean;
}

// CTAs of the staged even step: as many as fit on the SMs at once, found
// once per storage format
template <typename S>
static int staged_pair_blocks() {
    static int blocks = 0;
    if (blocks == 0) {
        const int smem = StagedPairLayout<S>::SMEM;
        cudaFuncSetAttribute(k_liquid_staged_pair<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        int per_sm = 0, dev = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_liquid_staged_pair<S>, SP_TILE / 2, smem);
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        blocks = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    }
    return blocks;
}

// blocks of the link pass: one resident wave (the kernel strides over the
// list), found once per storage format and parity
template <typename S, int PAR>
static int link_blocks() {
    static int blocks = 0;
    if (blocks == 0) {
        int per_sm = 0, dev = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solid_links<S, PAR>, 256, 0);
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        blocks = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    }
    return blocks;
}

// blocks of the bed kernel: one resident wave (the kernel strides over the
// list of bed segments)
template <typename S, int PAR>
static int bed_blocks() {
    static int blocks = 0;
    if (blocks == 0) {
        int per_sm = 0, dev = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_liquid_pair_bed<S, PAR>, 128, 0);
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        blocks = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    }
    return blocks;
}

template <typename S>
static void launch_typed(const Dev& s, int parity, cudaStream_t st, cudaEvent_t links_done) {
    const int lb = 152 * 8;
    // the particle forces are complete after the link pass, or with fluid-side
    // links after the whole sweep
    const bool early = s.np > 0 && !s.links_fused;
    // liquid kernels: threads along x, blocks over the rows (y, z)
    const dim3 lgrid((unsigned)((s.nx + 255) / 256), (unsigned)(s.ny * s.nz < 65535 ? s.ny * s.nz : 65535));
    if (parity == 0) {
        if (s.np > 0 && !s.links_fused) k_solid_links<S, 0><<<link_blocks<S, 0>(), 256, 0, st>>>(s);
        if (early && links_done) cudaEventRecord(links_done, st);
        if (use_staged_pairs(s)) {
            if constexpr (sizeof(S) == 2) {
                cudaMemsetAsync(s.tile_count, 0, sizeof(int), st);
                k_sp_tiles<<<(unsigned)((s.n / SP_TILE + 255) / 256), 256, 0, st>>>(s);
                k_liquid_staged_pair<S><<<staged_pair_blocks<S>(), SP_TILE / 2, StagedPairLayout<S>::SMEM, st>>>(s);
            }
        } else if (use_pairs(s)) {
            k_liquid_pair<S, 0, 0><<<lgrid, 128, 0, st>>>(s);
        } else {
            k_liquid<S, 0><<<lgrid, 256, 0, st>>>(s);
        }
        if (s.np > 0 && s.links_fused) k_liquid_pair_bed<S, 0><<<bed_blocks<S, 0>(), 128, 0, st>>>(s);
        k_interface<S, 0><<<lb, 128, 0, st>>>(s);
    } else {
        if (s.np > 0 && !s.links_fused) k_solid_links<S, 1><<<link_blocks<S, 1>(), 256, 0, st>>>(s);
        if (early && links_done) cudaEventRecord(links_done, st);
        if (use_split(s)) {
            k_liquid_pair<S, 1, 1><<<lgrid, 128, 0, st>>>(s);
            const long long ne = (2LL * s.nz + 2LL * (s.ny > 2 ? s.ny - 2 : 0)) * (s.nx / 2) +
                                 2LL * (s.ny > 2 ? s.ny - 2 : 0) * (s.nz > 2 ? s.nz - 2 : 0);
            k_liquid_pair_edges<S><<<blocks_for(ne, 128), 128, 0, st>>>(s);
        } else if (use_pairs(s)) {
            k_liquid_pair<S, 1, 0><<<lgrid, 128, 0, st>>>(s);
        } else {
            k_liquid<S, 1><<<lgrid, 256, 0, st>>>(s);
        }
        if (s.np > 0 && s.links_fused) k_liquid_pair_bed<S, 1><<<bed_blocks<S, 1>(), 128, 0, st>>>(s);
        k_interface<S, 1><<<lb, 128, 0, st>>>(s);
    }
    if (!early && links_done) cudaEventRecord(links_done, st);
}

int launch_stream_collide(const Dev& s, int parity, cudaStream_t st, cudaEvent_t links_done) {
    if (s.storage == FSLBM_STORE_FP32) launch_typed<float>(s, parity, st, links_done);
    else if (s.storage == FSLBM_STORE_FP16) launch_typed<__half>(s, parity, st, links_done);
    else launch_typed<__nv_bfloat16>(s, parity, st, links_done);
    const bool staged = parity == 0 && use_staged_pairs(s);
    const bool split = parity == 1 && use_split(s);
    return (s.np > 0 ? 1 : 0) + 2 + (staged ? 1 : 0) + (split ? 1 : 0);
}

}  // namespace fsl
