// step_kernels.cuh -- device code shared by the batched preparation (batch.cu)
// and the device-resident step (solver.cu): the per-element gather + rows of
// Eq. 1-4 (Sec. 2.4), the scatter onto the pleural mask, and the phases of
// the extraction (Sec. 2.3) run by every CTA of a cooperative grid.
#pragma once

#include <climits>

#include "mpm_internal.cuh"

namespace mpm {

struct BatchSys {
    BoxGeo g;
    int64_t NE;
    const int32_t *tile_coord;
    const int32_t *cell_id;     // lattice
    const uint8_t *mask;        // lattice
    const double *dfac_lat;     // lattice, or null
    double *field[kMaxSpecies]; // lattice fields (read by the preparation, written by the scatter)
    uint8_t *flags;
    int32_t *cell;
    double *dfac;
    double *x[kMaxSpecies], *cn[kMaxSpecies], *b[kMaxSpecies], *diag[kMaxSpecies];
    float *diag32[kMaxSpecies];
    int32_t *err;
    const int32_t *tile_index;  // device-resident step: the neighbour table is built here
    int32_t *nbr;
    const double *dk, *dq;      // device-resident step: per (species, cell) 1 + dt (mu + k), dt q
    AsmCoef C;
};

// Per-CTA tables of the device-resident preparation (uniform D): a D_s n for
// n open faces plus box faces counted twice (0..12), and 2 a D_s c_bc,s n
// for n box faces (0..6).
struct RowTab {
    double aDn[kMaxSpecies][13];
    double wbn[kMaxSpecies][7];
};

// Box cadence of the device-resident step (Sec. 2.3 refreshes the box every
// 50 MCS and keeps it in between).  Device memory, zero when the step is set
// up: refresh_ok = 1 lets the next step keep the box, count = steps since the
// last full extraction, guard_hit = a tumour voxel was gathered in the guard
// band, nfull = full extractions so far.
struct StepCad {
    uint32_t refresh_ok, count, guard_hit, nfull;
};

// The guard band of a box: the voxels within h of a box face that lies
// inside the lattice (a face on the lattice boundary cannot be crossed).
struct GuardBand {
    int h;
    int lo_in[3], hi_in[3];
    __device__ __forceinline__ bool in(int bx, int by, int bz, const BoxGeo &g) const
    {
        const int c[3] = {bx, by, bz};
        bool r = false;
#pragma unroll
        for (int d = 0; d < 3; ++d) r |= (lo_in[d] && c[d] < h) || (hi_in[d] && c[d] >= g.n[d] - h);
        return r;
    }
};

// One element of the fused preparation: flags, cell id, diffusivity factor
// and c^n gathered from the lattice, then the row of every species.
// kTab: the device-resident form (rows from the rate tables; tile coordinates
// and tables written earlier in the same kernel, so read through L2).
// gb (device-resident step): a tumour voxel in the guard band sets *hit.
template <bool kTab>
__device__ __forceinline__ void prep_elem(const BatchSys &S, const BoxGeo &g, int64_t e, const RowTab *tab = nullptr,
                                          const GuardBand *gb = nullptr, bool *hit = nullptr)
{
    const int ns = S.C.nspecies;
    int bx, by, bz;
    if (!elem_box<kTab>(e, g, S.tile_coord, bx, by, bz)) {   // tile padding
        S.flags[e] = 0;
        S.cell[e] = 0;
        if (S.dfac) S.dfac[e] = 1.0;
        for (int s = 0; s < ns; ++s) {
            S.x[s][e] = 0.0;
            S.cn[s][e] = 0.0;
            S.diag[s][e] = 1.0;
            S.diag32[s][e] = 1.0f;
            S.b[s][e] = 0.0;
        }
        return;
    }
    const int64_t sy = g.Lx, sz = (int64_t)g.Lx * g.Ly;
    const int64_t L = (int64_t)(g.lo[0] + bx) + sy * (g.lo[1] + by) + sz * (g.lo[2] + bz);
    // every lattice load of the element before its first store (a store may
    // alias a later load in the compiler's eyes): the mask at the voxel and
    // its in-box neighbours, the cell id, the diffusivity factor, c^n of
    // every species
    const bool hx0 = bx > 0, hx1 = bx < g.n[0] - 1, hy0 = by > 0, hy1 = by < g.n[1] - 1, hz0 = bz > 0,
               hz1 = bz < g.n[2] - 1;
    const uint32_t m0 = __ldg(S.mask + L);
    const uint32_t m1 = hx0 ? __ldg(S.mask + L - 1) : 0u, m2 = hx1 ? __ldg(S.mask + L + 1) : 0u;
    const uint32_t m3 = hy0 ? __ldg(S.mask + L - sy) : 0u, m4 = hy1 ? __ldg(S.mask + L + sy) : 0u;
    const uint32_t m5 = hz0 ? __ldg(S.mask + L - sz) : 0u, m6 = hz1 ? __ldg(S.mask + L + sz) : 0u;
    const int32_t id0 = __ldg(S.cell_id + L);
    if (gb && id0 > 0 && gb->in(bx, by, bz, g)) *hit = true;
    const double fp = S.dfac_lat ? __ldg(S.dfac_lat + L) : 1.0;
    double cs[kMaxSpecies];
#pragma unroll
    for (int s = 0; s < kMaxSpecies; ++s) cs[s] = s < ns ? __ldg(S.field[s] + L) : 0.0;
    uint32_t f = F_BOX;
    if (m0) {
        f |= F_MASK;
        if (m1) f |= F_MX;
        if (m2) f |= F_PX;
        if (m3) f |= F_MY;
        if (m4) f |= F_PY;
        if (m5) f |= F_MZ;
        if (m6) f |= F_PZ;
    }
    const bool inm = (f & F_MASK) != 0;
    const bool bad = inm && (id0 < 0 || id0 >= S.C.ncell);
    const int32_t id = bad ? 0 : id0;
    // the rate-table entries of the cell id, every species together
    double dkv[kMaxSpecies], dqv[kMaxSpecies];
    const bool tabrow = kTab && !S.dfac && inm;
#pragma unroll
    for (int s = 0; s < kMaxSpecies; ++s) {
        const int64_t k = (int64_t)s * S.C.ncell + id;
        dkv[s] = tabrow && s < ns ? __ldcg(S.dk + k) : 0.0;
        dqv[s] = tabrow && s < ns ? __ldcg(S.dq + k) : 0.0;
    }
    S.flags[e] = (uint8_t)f;
    S.cell[e] = id0;
    if (S.dfac) S.dfac[e] = fp;
    if (bad) atomicOr(S.err, 1);
    if (!inm) {                                 // identity row keeping c^n
#pragma unroll
        for (int s = 0; s < kMaxSpecies; ++s) {
            if (s >= ns) break;
            const double c = cs[s];
            S.x[s][e] = c;
            S.cn[s][e] = c;
            S.diag[s][e] = 1.0;
            S.diag32[s][e] = 1.0f;
            S.b[s][e] = c;
        }
        return;
    }
    const int ndir = S.C.bc_box == 0 ? (bx == 0) + (bx == g.n[0] - 1) + (by == 0) + (by == g.n[1] - 1) +
                                           (bz == 0) + (bz == g.n[2] - 1)
                                     : 0;
    auto dq = [&](int d) -> double {
        const int64_t o = d == 0 ? -1 : d == 1 ? 1 : d == 2 ? -sy : d == 3 ? sy : d == 4 ? -sz : sz;
        return __ldg(S.dfac_lat + L + o);
    };
#pragma unroll
    for (int s = 0; s < kMaxSpecies; ++s) {
        if (s >= ns) break;
        const double c = cs[s];
        double dg, bb;
        if (tabrow) {
            // the rows of assemble_row with the per-cell and per-count products
            // taken from tables: three FP64 additions per species
            dg = dkv[s] + tab->aDn[s][__popc(f & F_OPEN) + 2 * ndir];
            bb = (c + dqv[s]) + tab->wbn[s][ndir];
        } else {
            assemble_row(S.C, s, f, id, ndir, S.dfac != nullptr, fp, dq, c, dg, bb);
        }
        S.x[s][e] = c;
        S.cn[s][e] = c;
        S.diag[s][e] = dg;
        S.diag32[s][e] = f32_rz(dg);
        S.b[s][e] = bb;
    }
}

// The device-resident preparation for uniform D on tiles at least four wide
// in x: one 4-element chunk of a tile row (four x-consecutive voxels of the
// lattice) per call.  One tile-coordinate load serves the four elements, the
// lattice loads of all four are in flight together, and the element arrays
// are written with 4- to 16-byte stores.  Per element the rows are those of
// prep_elem<true> (same operands, same order).
__device__ __forceinline__ void prep_chunk(const BatchSys &S, const BoxGeo &g, uint32_t r, const RowTab *tab,
                                           const GuardBand *gb, bool *hit)
{
    const int ns = S.C.nspecies;
    const uint32_t e = r << 2;
    const int ltv = g.lt[0] + g.lt[1] + g.lt[2];
    const int4 tc = __ldcg(reinterpret_cast<const int4 *>(S.tile_coord) + (e >> ltv));
    const uint32_t v0 = e & ((1u << ltv) - 1u);
    const int ix0 = (int)(v0 & ((1u << g.lt[0]) - 1u));
    const int iy = (int)((v0 >> g.lt[0]) & ((1u << g.lt[1]) - 1u)), iz = (int)(v0 >> (g.lt[0] + g.lt[1]));
    const int bx0 = (tc.x << g.lt[0]) + ix0, by = (tc.y << g.lt[1]) + iy, bz = (tc.z << g.lt[2]) + iz;
    const int nv = (by < g.n[1] && bz < g.n[2]) ? max(0, min(4, g.n[0] - bx0)) : 0;   // elements in the box
    const int64_t sy = g.Lx, sz = (int64_t)g.Lx * g.Ly;
    const int64_t L0 = (int64_t)(g.lo[0] + bx0) + sy * (g.lo[1] + by) + sz * (g.lo[2] + bz);
    const bool hy0 = by > 0, hy1 = by < g.n[1] - 1, hz0 = bz > 0, hz1 = bz < g.n[2] - 1;
    uint32_t mo[4], my0[4], my1[4], mz0[4], mz1[4];
    int32_t id0[4];
    double cs[kMaxSpecies][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const bool in = k < nv;
        const int64_t L = L0 + k;
        mo[k] = in ? __ldg(S.mask + L) : 0u;
        my0[k] = in && hy0 ? __ldg(S.mask + L - sy) : 0u;
        my1[k] = in && hy1 ? __ldg(S.mask + L + sy) : 0u;
        mz0[k] = in && hz0 ? __ldg(S.mask + L - sz) : 0u;
        mz1[k] = in && hz1 ? __ldg(S.mask + L + sz) : 0u;
        id0[k] = in ? __ldg(S.cell_id + L) : 0;
#pragma unroll
        for (int s = 0; s < kMaxSpecies; ++s) cs[s][k] = in && s < ns ? __ldg(S.field[s] + L) : 0.0;
    }
    if (gb) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (k < nv && id0[k] > 0 && gb->in(bx0 + k, by, bz, g)) *hit = true;
    }
    const uint32_t mxm = nv > 0 && bx0 > 0 ? __ldg(S.mask + L0 - 1) : 0u;
    const uint32_t mxp = nv == 4 && bx0 + 4 < g.n[0] ? __ldg(S.mask + L0 + 4) : 0u;
    uint32_t f[4];
    int32_t id[4];
    int nd[4];
    bool anybad = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int bx = bx0 + k;
        uint32_t fk = k < nv ? F_BOX : 0u;
        if (mo[k]) {
            fk |= F_MASK;
            if (k > 0 ? mo[k - 1] != 0u : mxm != 0u) fk |= F_MX;
            if (k < 3 ? (k + 1 < nv && mo[k + 1] != 0u) : mxp != 0u) fk |= F_PX;
            if (my0[k]) fk |= F_MY;
            if (my1[k]) fk |= F_PY;
            if (mz0[k]) fk |= F_MZ;
            if (mz1[k]) fk |= F_PZ;
        }
        f[k] = fk;
        const bool bad = (fk & F_MASK) && (id0[k] < 0 || id0[k] >= S.C.ncell);
        anybad |= bad;
        id[k] = bad ? 0 : id0[k];
        nd[k] = S.C.bc_box == 0 ? (bx == 0) + (bx == g.n[0] - 1) + (by == 0) + (by == g.n[1] - 1) + (bz == 0) +
                                      (bz == g.n[2] - 1)
                                : 0;
    }
    *reinterpret_cast<uchar4 *>(S.flags + e) = make_uchar4((uint8_t)f[0], (uint8_t)f[1], (uint8_t)f[2], (uint8_t)f[3]);
    *reinterpret_cast<int4 *>(S.cell + e) = make_int4(id0[0], id0[1], id0[2], id0[3]);
    if (anybad) atomicOr(S.err, 1);
#pragma unroll
    for (int s = 0; s < kMaxSpecies; ++s) {
        if (s >= ns) break;
        double dkv[4], dqv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t t = (int64_t)s * S.C.ncell + id[k];
            const bool row = (f[k] & F_MASK) != 0;
            // plain cached loads: the tables were written before a grid barrier
            // and never read before it, and neighbouring voxels mostly share a cell
            dkv[k] = row ? S.dk[t] : 0.0;
            dqv[k] = row ? S.dq[t] : 0.0;
        }
        double xo[4], dg[4], bb[4];
        float d32[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const double c = cs[s][k];
            if (!(f[k] & F_BOX)) {            // tile padding
                xo[k] = 0.0;
                dg[k] = 1.0;
                bb[k] = 0.0;
            } else if (!(f[k] & F_MASK)) {    // identity row keeping c^n
                xo[k] = c;
                dg[k] = 1.0;
                bb[k] = c;
            } else {
                xo[k] = c;
                dg[k] = dkv[k] + tab->aDn[s][__popc(f[k] & F_OPEN) + 2 * nd[k]];
                bb[k] = (c + dqv[k]) + tab->wbn[s][nd[k]];
            }
            d32[k] = f32_rz(dg[k]);
        }
        double2 *x2 = reinterpret_cast<double2 *>(S.x[s] + e), *c2 = reinterpret_cast<double2 *>(S.cn[s] + e);
        double2 *b2 = reinterpret_cast<double2 *>(S.b[s] + e), *g2 = reinterpret_cast<double2 *>(S.diag[s] + e);
        x2[0] = make_double2(xo[0], xo[1]);
        x2[1] = make_double2(xo[2], xo[3]);
        c2[0] = make_double2(xo[0], xo[1]);
        c2[1] = make_double2(xo[2], xo[3]);
        b2[0] = make_double2(bb[0], bb[1]);
        b2[1] = make_double2(bb[2], bb[3]);
        g2[0] = make_double2(dg[0], dg[1]);
        g2[1] = make_double2(dg[2], dg[3]);
        *reinterpret_cast<float4 *>(S.diag32[s] + e) = make_float4(d32[0], d32[1], d32[2], d32[3]);
    }
}

// The scatter on a 4-element chunk of a tile row (one tile-coordinate load
// and one flags word for four elements).  The tile coordinates were written
// earlier in the same kernel.
__device__ __forceinline__ void scatter_chunk(const BatchSys &S, const BoxGeo &g, uint32_t r)
{
    const uint32_t e = r << 2;
    const uchar4 fl = *reinterpret_cast<const uchar4 *>(S.flags + e);
    const uint32_t f[4] = {fl.x, fl.y, fl.z, fl.w};
    if (!((f[0] | f[1] | f[2] | f[3]) & F_MASK)) return;
    const int ltv = g.lt[0] + g.lt[1] + g.lt[2];
    const int4 tc = __ldcg(reinterpret_cast<const int4 *>(S.tile_coord) + (e >> ltv));
    const uint32_t v0 = e & ((1u << ltv) - 1u);
    const int bx0 = (tc.x << g.lt[0]) + (int)(v0 & ((1u << g.lt[0]) - 1u));
    const int by = (tc.y << g.lt[1]) + (int)((v0 >> g.lt[0]) & ((1u << g.lt[1]) - 1u));
    const int bz = (tc.z << g.lt[2]) + (int)(v0 >> (g.lt[0] + g.lt[1]));
    const int64_t L0 =
        (int64_t)(g.lo[0] + bx0) + (int64_t)g.Lx * ((g.lo[1] + by) + (int64_t)g.Ly * (g.lo[2] + bz));
    for (int s = 0; s < S.C.nspecies; ++s) {
        const double2 a = reinterpret_cast<const double2 *>(S.x[s] + e)[0];
        const double2 c = reinterpret_cast<const double2 *>(S.x[s] + e)[1];
        const double xv[4] = {a.x, a.y, c.x, c.y};
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (f[k] & F_MASK) S.field[s][L0 + k] = xv[k];
    }
}

// Sec. 2.4: the box solution onto the pleural mask (in-mask voxels only).
// kCoherent: the tile coordinates were written earlier in the same kernel.
template <bool kCoherent = false>
__device__ __forceinline__ void scatter_elem(const BatchSys &S, const BoxGeo &g, int64_t e)
{
    if (!(S.flags[e] & F_MASK)) return;
    int bx, by, bz;
    elem_box<kCoherent>(e, g, S.tile_coord, bx, by, bz);
    const int64_t L = (int64_t)(g.lo[0] + bx) + (int64_t)g.Lx * ((g.lo[1] + by) + (int64_t)g.Ly * (g.lo[2] + bz));
    for (int s = 0; s < S.C.nspecies; ++s) S.field[s][L] = S.x[s][e];
}

// Per-(species, cell) rate terms of the rows (Eq. 1-4) for the device-resident
// preparation: dk = 1 + dt (mu_s + k_cell[s][id]), dq = dt q_cell[s][id].
struct RateArgs {
    int32_t nspecies, ncell;
    double dt;
    double mu[kMaxSpecies];
    const double *k_cell, *q_cell;
    double *dk, *dq;
};

struct ExtractArgs {
    const int32_t *cell_id;
    const uint8_t *mask;
    int32_t L[3], lt[3], margin, vec4;
    int32_t *part_box;                 // [grid][8]: per-CTA min[3], max[3]
    unsigned long long *part_cnt;      // [grid][2]: per-CTA mask voxels, active tiles
    uint32_t *bar;                     // grid barrier counter (zero at launch)
    int32_t *xabort;                   // set when a grid barrier gave up
    uint64_t timeout_ns;
    int32_t *box_out;                  // raw min[3], max[3] (for the host)
    BoxGeo *geo_out;
    unsigned long long *count_out;     // mask voxels, active tiles (for the host)
    StepDyn *dyn;
    int8_t *active;
    int32_t *tile_index, *tile_coord, *err;
    uint32_t *sbar;                    // the solver's barrier counters and reports: zeroed here
    int32_t nsbar;
    uint32_t *srep;
    int32_t nrep_words;
    RateArgs ra;
    StepCad *cad;                      // box cadence state
    int32_t box_every, box_guard;      // mpm_opts' cadence: full extraction every box_every steps
    unsigned long long *prof;          // nullable: CTA 0 adds ns per phase A..E (each up to its barrier)
};

// Per-CTA row tables and, grid-strided, the per-(species, cell) rate tables.
template <int NT>
__device__ __forceinline__ void row_tables(const ExtractArgs &A, const BatchSys &S, int b, int nb, RowTab &tab)
{
    const int tid = threadIdx.x;
    for (int i = tid; i < S.C.nspecies * 20; i += NT) {
        const int s = i / 20, n = i % 20;
        if (n < 13) tab.aDn[s][n] = S.C.a * S.C.D[s] * (double)n;
        else tab.wbn[s][n - 13] = S.C.a * 2.0 * S.C.D[s] * S.C.cbc[s] * (double)(n - 13);
    }
    const int64_t nr = (int64_t)A.ra.nspecies * A.ra.ncell;
    for (int64_t i = (int64_t)b * NT + tid; i < nr; i += (int64_t)nb * NT) {
        const int s = (int)(i / A.ra.ncell);
        A.ra.dk[i] = 1.0 + A.ra.dt * (A.ra.mu[s] + A.ra.k_cell[i]);
        A.ra.dq[i] = A.ra.dt * A.ra.q_cell[i];
    }
}

// The guard band of box g (empty unless the cadence keeps boxes).
__device__ __forceinline__ GuardBand guard_band(const ExtractArgs &A, const BoxGeo &g)
{
    GuardBand gb;
    gb.h = A.box_every > 1 ? A.box_guard : 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        gb.lo_in[d] = g.lo[d] > 0;
        gb.hi_in[d] = g.lo[d] + g.n[d] < A.L[d];
    }
    return gb;
}

// Phase E: gather + rows of every stored element (4-element chunks where the
// tiles are at least four wide and D is uniform), the neighbour table when
// nbr, and with kGuard the guard vote (one atomic per CTA).
template <int NT, bool kGuard>
__device__ __forceinline__ void gather_phase_t(const ExtractArgs &A, const BatchSys &S, const BoxGeo &g, int64_t NE,
                                               int b, int nb, const RowTab &tab, bool nbr)
{
    const int tid = threadIdx.x;
    const int ltv = g.lt[0] + g.lt[1] + g.lt[2];
    const GuardBand gbv = guard_band(A, g);
    const GuardBand *gb = kGuard ? &gbv : nullptr;
    bool hit = false;
    const bool chunks = g.lt[0] >= 2 && !S.dfac;
    const int64_t nunit = chunks ? NE >> 2 : NE;   // 4-element chunks or elements
    for (int64_t u = (int64_t)b * NT + tid; u < nunit; u += (int64_t)nb * NT) {
        const int64_t e = chunks ? u << 2 : u;
        if (chunks) prep_chunk(S, g, (uint32_t)u, &tab, gb, &hit);
        else prep_elem<true>(S, g, e, &tab, gb, &hit);
        if (nbr && (e & ((1 << ltv) - 1)) == 0) {   // neighbour tiles of this tile
            const int64_t a = e >> ltv;
            const int4 c = __ldcg(reinterpret_cast<const int4 *>(S.tile_coord) + a);
#pragma unroll
            for (int d = 0; d < 6; ++d) {
                int32_t q[3] = {c.x, c.y, c.z};
                q[d >> 1] += (d & 1) ? 1 : -1;
                int32_t r = -1;
                if (q[0] >= 0 && q[0] < g.nt[0] && q[1] >= 0 && q[1] < g.nt[1] && q[2] >= 0 && q[2] < g.nt[2])
                    r = __ldcg(S.tile_index + (q[2] * g.nt[1] + q[1]) * g.nt[0] + q[0]);
                S.nbr[6 * a + d] = r;
            }
        }
    }
    if (kGuard && __syncthreads_or(hit) && tid == 0) atomicOr(&A.cad->guard_hit, 1u);
}

template <int NT>
__device__ __forceinline__ void gather_phase(const ExtractArgs &A, const BatchSys &S, const BoxGeo &g, int64_t NE,
                                             int b, int nb, const RowTab &tab, bool nbr)
{
    if (A.box_every > 1 && A.box_guard > 0) gather_phase_t<NT, true>(A, S, g, NE, b, nb, tab, nbr);
    else gather_phase_t<NT, false>(A, S, g, NE, b, nb, tab, nbr);
}

// Block-wide sum over NT threads (every thread gets the total).
template <int NT>
__device__ __forceinline__ unsigned long long xblock_sum(unsigned long long v, unsigned long long *sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    unsigned long long t = 0;
    for (int i = 0; i < NT / 32; ++i) t += sh[i];
    return t;
}

// The extraction and preparation of the device-resident step, run by every
// CTA of a cooperative grid of nb CTAs of NT threads: phases separated by
// bounded grid barriers (counter A.bar, epoch carried by the caller), partial
// results per CTA (no atomics, so every count is deterministic).
//   A  bounding box of cell_id > 0 (Sec. 2.3): per-CTA min / max
//   B  box from all partials (every CTA); tile activity of the box rows and
//      the in-mask count; rate tables
//   C  active tiles per CTA chunk of the box tiles
//   D  compaction: chunk offsets from the partial counts, compact index and
//      coordinates of every tile, activity bytes cleared for the next step;
//      the solver's barrier counters and reports zeroed
//   E  the gather and rows of every stored element (Eq. 1-4) and the tile
//      neighbour table; CTA 0 then publishes the box and element count.
// Returns false when a grid barrier gave up (A.xabort is then set).
template <int NT>
__device__ __forceinline__ bool extract_phases(const ExtractArgs &A, const BatchSys &S, int b, int nb,
                                               uint32_t &epoch)
{
    __shared__ int32_t smm[6][NT / 32];
    __shared__ unsigned long long ssum[NT / 32];
    __shared__ BoxGeo g;
    __shared__ RowTab tab;
    __shared__ int32_t wtot[NT / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool prof = A.prof != nullptr && b == 0 && tid == 0;
    uint64_t tp = prof ? globaltimer_ns() : 0;
    auto tick = [&](int slot) {
        if (prof) {
            const uint64_t t = globaltimer_ns();
            A.prof[slot] += t - tp;
            tp = t;
        }
    };
    if (b == 0 && tid == 0) {
        A.dyn->NE = 0;
        A.dyn->g.n[0] = 0;
        A.cad->guard_hit = 0u;
    }
    // ---- A: bounding box, per CTA
    {
        const int64_t Ltot = (int64_t)A.L[0] * A.L[1] * A.L[2];
        const uint32_t Lx = (uint32_t)A.L[0], Lxy = (uint32_t)(A.L[0] * A.L[1]);
        int mn[3] = {INT_MAX, INT_MAX, INT_MAX}, mx[3] = {-1, -1, -1};
        const uint32_t t0 = b * NT + tid, nth = nb * NT;
        uint32_t done = 0;
        if (A.vec4) {
            const int4 *c4 = reinterpret_cast<const int4 *>(A.cell_id);
            const uint32_t n4 = (uint32_t)(Ltot / 4);
            // 16-byte streaming loads, kD per thread in flight (about 64 KB per
            // SM): the scan is bound by the bytes the SMs keep in flight
            constexpr int kD = NT <= 512 ? 8 : 4;
            const bool rows4 = (Lx & 3u) == 0;   // the four voxels of a load share a row
            uint32_t q = t0;
            for (; q + (kD - 1) * nth < n4; q += kD * nth) {
                int4 v[kD];
#pragma unroll
                for (int u = 0; u < kD; ++u) v[u] = __ldcs(c4 + q + u * nth);
#pragma unroll
                for (int u = 0; u < kD; ++u) {
                    const uint32_t pm = (v[u].x > 0) | ((v[u].y > 0) << 1) | ((v[u].z > 0) << 2) | ((v[u].w > 0) << 3);
                    if (!pm) continue;
                    const uint32_t e = 4 * (q + u * nth);
                    if (rows4) {   // the first and the last tumour voxel bound the other two
                        bbox_upd(e + (__ffs(pm) - 1), Lx, Lxy, mn, mx);
                        bbox_upd(e + (31 - __clz(pm)), Lx, Lxy, mn, mx);
                    } else {
                        if (pm & 1u) bbox_upd(e + 0, Lx, Lxy, mn, mx);
                        if (pm & 2u) bbox_upd(e + 1, Lx, Lxy, mn, mx);
                        if (pm & 4u) bbox_upd(e + 2, Lx, Lxy, mn, mx);
                        if (pm & 8u) bbox_upd(e + 3, Lx, Lxy, mn, mx);
                    }
                }
            }
            for (; q < n4; q += nth) {
                const int4 v = __ldcs(c4 + q);
                const uint32_t e = 4 * q;
                if (v.x > 0) bbox_upd(e + 0, Lx, Lxy, mn, mx);
                if (v.y > 0) bbox_upd(e + 1, Lx, Lxy, mn, mx);
                if (v.z > 0) bbox_upd(e + 2, Lx, Lxy, mn, mx);
                if (v.w > 0) bbox_upd(e + 3, Lx, Lxy, mn, mx);
            }
            done = n4 * 4;
        }
        for (uint32_t e = done + t0; e < (uint32_t)Ltot; e += nth)
            if (__ldcs(A.cell_id + e) > 0) bbox_upd(e, Lx, Lxy, mn, mx);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int lo = __reduce_min_sync(0xffffffffu, mn[d]);
            const int hi = __reduce_max_sync(0xffffffffu, mx[d]);
            if (lane == 0) { smm[d][warp] = lo; smm[3 + d][warp] = hi; }
        }
        __syncthreads();
        if (tid < 6) {
            int v = tid < 3 ? INT_MAX : -1;
            for (int i = 0; i < NT / 32; ++i) v = tid < 3 ? min(v, smm[tid][i]) : max(v, smm[tid][i]);
            A.part_box[8 * b + tid] = v;
        }
    }
    if (!team_barrier(A.bar, epoch, nb, A.xabort, A.timeout_ns)) return false;
    tick(10);
    // ---- B: the box (every CTA), tile activity, in-mask count, rate tables
    {
        int mn[3] = {INT_MAX, INT_MAX, INT_MAX}, mx[3] = {-1, -1, -1};
        for (int i = tid; i < nb; i += NT) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                mn[d] = min(mn[d], __ldcg(A.part_box + 8 * i + d));
                mx[d] = max(mx[d], __ldcg(A.part_box + 8 * i + 3 + d));
            }
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int lo = __reduce_min_sync(0xffffffffu, mn[d]);
            const int hi = __reduce_max_sync(0xffffffffu, mx[d]);
            if (lane == 0) { smm[d][warp] = lo; smm[3 + d][warp] = hi; }
        }
        __syncthreads();
        if (tid == 0) {
            int32_t mm[6];
            for (int d = 0; d < 6; ++d) {
                int v = d < 3 ? INT_MAX : -1;
                for (int i = 0; i < NT / 32; ++i) v = d < 3 ? min(v, smm[d][i]) : max(v, smm[d][i]);
                mm[d] = v;
            }
            g = box_geo(mm, A.margin, A.L[0], A.L[1], A.L[2], A.lt[0], A.lt[1], A.lt[2]);
            if (b == 0) {
                for (int d = 0; d < 6; ++d) A.box_out[d] = mm[d];
                *A.geo_out = g;
            }
        }
        row_tables<NT>(A, S, b, nb, tab);   // per-CTA row tables (phase E), rate tables
        __syncthreads();
        unsigned long long cnt = 0;
        if (g.n[0] > 0) {
            // one row of tiles (TY x TZ box rows) per warp and iteration: for
            // each 32-voxel chunk the mask bytes of those rows are in flight
            // together and OR-ed, and the chunk's active tiles are written
            // once, by the first lane of each tile (the rows of a tile would
            // otherwise store the same activity bytes again and again)
            const int64_t gw = (int64_t)b * (NT / 32) + warp, nw = (int64_t)nb * (NT / 32);
            const int TX = 1 << g.lt[0], TY = 1 << g.lt[1], TZ = 1 << g.lt[2];
            const int64_t ngroups = (int64_t)g.nt[1] * g.nt[2];
            for (int64_t grp = gw; grp < ngroups; grp += nw) {
                const int ty = (int)(grp % g.nt[1]), tz = (int)(grp / g.nt[1]);
                const int64_t trow = ((int64_t)tz * g.nt[1] + ty) * g.nt[0];
                const int y1 = min(TY, g.n[1] - ty * TY), z1 = min(TZ, g.n[2] - tz * TZ);
                const int nr = y1 * z1;
                for (int c0 = 0; c0 < g.n[0]; c0 += 32) {
                    const int bx = c0 + lane;
                    uint32_t any = 0u;
                    if (bx < g.n[0]) {
#pragma unroll 4
                        for (int r = 0; r < nr; ++r) {
                            const int by = ty * TY + r % y1, bz = tz * TZ + r / y1;
                            const int64_t L0 = (int64_t)g.lo[0] +
                                               (int64_t)g.Lx * ((int64_t)(g.lo[1] + by) + (int64_t)g.Ly * (g.lo[2] + bz));
                            const uint32_t m = __ldg(A.mask + L0 + bx);
                            cnt += m != 0u ? 1u : 0u;
                            any |= m;
                        }
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, any != 0u);
                    if ((lane & (TX - 1)) == 0 && ((bal >> lane) & ((TX >= 32) ? 0xffffffffu : ((1u << TX) - 1u))))
                        A.active[trow + (bx >> g.lt[0])] = 1;
                }
            }
        }
        cnt = xblock_sum<NT>(cnt, ssum);
        if (tid == 0) A.part_cnt[2 * b + 0] = cnt;
    }
    if (!team_barrier(A.bar, epoch, nb, A.xabort, A.timeout_ns)) return false;
    tick(11);
    // ---- C: active tiles of this CTA's chunk (8-tile words)
    const int32_t ntiles = g.n[0] > 0 ? g.nt[0] * g.nt[1] * g.nt[2] : 0;
    const int32_t nwords = (ntiles + 7) >> 3;
    const int32_t wchunk = (nwords + nb - 1) / nb;
    const int32_t w0 = min(nwords, b * wchunk), w1 = min(nwords, w0 + wchunk);
    unsigned long long *aw = reinterpret_cast<unsigned long long *>(A.active);
    auto word = [&](int32_t wi) -> unsigned long long {
        unsigned long long w = __ldcg(aw + wi);
        const int32_t i0 = 8 * wi;
        if (i0 + 8 > ntiles) w &= ~0ull >> (8 * (i0 + 8 - ntiles));
        return w;
    };
    // up to 8192 words (64 Ki tiles) every CTA counts the active tiles before
    // its chunk itself, which spares this phase and its grid barrier
    const bool onepass = nwords <= 8192;
    if (!onepass) {
        unsigned long long c = 0;
        for (int32_t wi = w0 + tid; wi < w1; wi += NT) c += __popcll(word(wi) & 0x0101010101010101ull);
        c = xblock_sum<NT>(c, ssum);
        if (tid == 0) A.part_cnt[2 * b + 1] = c;
        if (!team_barrier(A.bar, epoch, nb, A.xabort, A.timeout_ns)) return false;
    }
    tick(12);
    // ---- D: compaction
    int64_t nact = 0;
    {
        unsigned long long before = 0, tot = 0, mtot = 0;
        for (int i = tid; i < nb; i += NT) {
            if (!onepass) {
                const unsigned long long c = __ldcg(A.part_cnt + 2 * i + 1);
                tot += c;
                if (i < b) before += c;
            }
            mtot += __ldcg(A.part_cnt + 2 * i + 0);
        }
        if (onepass) {
            for (int32_t wi = tid; wi < nwords; wi += NT) {
                const unsigned long long c = __popcll(word(wi) & 0x0101010101010101ull);
                tot += c;
                if (wi < w0) before += c;
            }
        }
        before = xblock_sum<NT>(before, ssum);
        tot = xblock_sum<NT>(tot, ssum);
        mtot = xblock_sum<NT>(mtot, ssum);
        nact = (int64_t)tot;
        if (b == 0 && tid == 0) {
            A.count_out[0] = mtot;
            A.count_out[1] = tot;
            *A.err = 0;
        }
        if (b == 0) {
            for (int i = tid; i < A.nsbar; i += NT) A.sbar[i] = 0u;
            for (int i = tid; i < A.nrep_words; i += NT) A.srep[i] = 0u;
        }
        const int32_t nxy = g.nt[0] * g.nt[1];
        int32_t carry = (int32_t)before;
        for (int32_t base = w0; base < w1; base += NT) {
            const int32_t wi = base + tid;
            const unsigned long long w = wi < w1 ? word(wi) : 0ull;
            const int32_t c = __popcll(w & 0x0101010101010101ull);
            int32_t incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            __syncthreads();
            if (lane == 31) wtot[warp] = incl;
            __syncthreads();
            int32_t woff = 0, rtot = 0;
            for (int i = 0; i < NT / 32; ++i) {
                const int32_t t = wtot[i];
                if (i < warp) woff += t;
                rtot += t;
            }
            int32_t idx = carry + woff + incl - c;
            if (wi < w1) {
                const int32_t i0 = 8 * wi;
                int32_t tx = i0 % g.nt[0], ty = (i0 / g.nt[0]) % g.nt[1], tz = i0 / nxy;
                for (int k = 0; k < 8; ++k) {
                    const int32_t i = i0 + k;
                    if (i >= ntiles) break;
                    if ((w >> (8 * k)) & 1ull) {
                        A.tile_index[i] = idx;
                        reinterpret_cast<int4 *>(A.tile_coord)[idx] = make_int4(tx, ty, tz, 0);
                        ++idx;
                    } else {
                        A.tile_index[i] = -1;
                    }
                    if (++tx == g.nt[0]) {
                        tx = 0;
                        if (++ty == g.nt[1]) { ty = 0; ++tz; }
                    }
                }
            }
            carry += rtot;
        }
    }
    if (!team_barrier(A.bar, epoch, nb, A.xabort, A.timeout_ns)) return false;
    tick(13);
    // ---- E: gather + rows of every stored element, neighbour table
    // (the activity words of this CTA's chunk are cleared for the next step
    // here, after every CTA has counted them)
    for (int32_t wi = w0 + tid; wi < w1; wi += NT) aw[wi] = 0ull;
    const int ltv = g.lt[0] + g.lt[1] + g.lt[2];
    const int64_t NE = g.n[0] > 0 ? nact << ltv : 0;
    gather_phase<NT>(A, S, g, NE, b, nb, tab, true);
    if (b == 0 && tid == 0) {
        A.dyn->g = g;
        A.dyn->NE = NE;
    }
    tick(14);
    return true;
}

// A step that keeps the box, tiles and neighbour table of the last full
// extraction (box_every > 1): the resets the compaction does, the row and rate
// tables, one grid barrier, then the gather + rows of every stored element.
template <int NT>
__device__ __forceinline__ bool refresh_phases(const ExtractArgs &A, const BatchSys &S, int b, int nb, uint32_t &epoch)
{
    __shared__ RowTab tab;
    const int tid = threadIdx.x;
    const bool prof = A.prof != nullptr && b == 0 && tid == 0;
    uint64_t tp = prof ? globaltimer_ns() : 0;
    if (b == 0) {
        if (tid == 0) {
            *A.err = 0;
            A.cad->guard_hit = 0u;
        }
        for (int i = tid; i < A.nsbar; i += NT) A.sbar[i] = 0u;
        for (int i = tid; i < A.nrep_words; i += NT) A.srep[i] = 0u;
    }
    row_tables<NT>(A, S, b, nb, tab);
    __syncthreads();
    if (!team_barrier(A.bar, epoch, nb, A.xabort, A.timeout_ns)) return false;
    const BoxGeo g = A.dyn->g;
    const int64_t NE = A.dyn->NE;
    gather_phase<NT>(A, S, g, NE, b, nb, tab, false);
    if (prof) A.prof[14] += globaltimer_ns() - tp;
    return true;
}


}  // namespace mpm
