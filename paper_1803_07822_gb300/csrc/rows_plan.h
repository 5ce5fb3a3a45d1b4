// Shape of the row-staged step pass (host and device): tile size, the byte
// layout of one shared-memory stage, and whether the pass applies.
#pragma once

namespace cslbm {
namespace rows {

constexpr int NT = 256;        // compute threads of a CTA, nodes of a tile at most
constexpr int NW = NT / 32;    // compute warps
constexpr int NTHR = NT + 32;  // + the copy warp
constexpr int STAGES = 2;
constexpr int NGEO = 25, NHIST = 10;
// limit of every wait of the row-staged and fused passes (half a second)
constexpr unsigned long long kWaitNs = 500000000ull;

// A tile is TR whole x-rows of one plane.  In a stage the populations sit at
// [lambda][NT], rho u at [z-layer][JS] (16-byte nodes), geometry at
// [25][NT] and history at [10][NT], every block 128-byte aligned.
struct Plan {
    int TR;        // rows per tile
    int nyb;       // tiles per plane
    int y1;        // first row of the first tile: 1 when tiles are single rows and axis 1 is
                   // not periodic (the face rows, stepped by the face pass, get no tile)
    int z0;        // first plane that is not a face plane
    int ntiles;    // nyb * (planes that are not face planes)
    int JS;        // nodes per rho u layer: (TR + 2) n0 rounded up to 8
    int JL;        // floats per line of the 2-D view of rho u: the largest power
                   // of two <= 256 dividing 4 n0
    int JR;        // lines of one rho u layer: (TR + 2) 4 n0 / JL
    unsigned off_jf, off_geo, off_hist, stage_bytes;
};

inline unsigned smem_bytes(const Plan& pl) { return STAGES * pl.stage_bytes + 2 * STAGES * 8; }

// false when the pass does not apply: rows longer than NT nodes or not a
// whole number of 16-byte chunks, fewer than NT nodes in all, or stages that
// do not fit in max_smem bytes
inline bool make_plan(const int n[3], bool yper, bool zper, int s_bytes, int max_smem, Plan& pl)
{
    const long long N = (long long)n[0] * n[1] * n[2];
    if (n[0] > NT || n[0] % 4 != 0 || (n[0] * s_bytes) % 16 != 0 || N < NT) return false;
    if (!zper && n[2] < 3) return false;
    if (!yper && n[1] < 3) return false;
    pl.TR = NT / n[0] < n[1] ? NT / n[0] : n[1];
    pl.y1 = (pl.TR == 1 && !yper) ? 1 : 0;
    pl.nyb = pl.y1 ? n[1] - 2 : (n[1] + pl.TR - 1) / pl.TR;
    pl.z0 = zper ? 0 : 1;
    pl.ntiles = pl.nyb * (zper ? n[2] : n[2] - 2);
    pl.JS = ((pl.TR + 2) * n[0] + 7) / 8 * 8;
    pl.JL = 256;
    while ((4 * n[0]) % pl.JL != 0) pl.JL /= 2;
    pl.JR = (pl.TR + 2) * 4 * n[0] / pl.JL;
    unsigned o = ((unsigned)(19 * NT * s_bytes) + 127u) & ~127u;
    pl.off_jf = o;
    o += 3u * pl.JS * 16u;
    o = (o + 127u) & ~127u;
    pl.off_geo = o;
    o += NGEO * NT * 4u;
    pl.off_hist = o;
    o += NHIST * NT * 4u;
    pl.stage_bytes = (o + 127u) & ~127u;
    return (long long)smem_bytes(pl) <= max_smem;
}

// smem layout of the fused pass after the two step stages: the momentum
// stage (populations, sqrt(g), A and B; off_sg and off_h4 relative to it),
// two rho u tiles of NT nodes, then ten mbarriers; false when it does not fit
inline bool fused_layout(const Plan& pl, int s_bytes, int max_smem, unsigned& off_m, unsigned& off_sg,
                         unsigned& off_h4, unsigned& off_js, unsigned& bytes)
{
    off_m = 2u * pl.stage_bytes;
    off_sg = ((unsigned)(19 * NT * s_bytes) + 127u) & ~127u;
    off_h4 = off_sg + NT * 4u;
    off_js = off_m + ((off_h4 + 4u * NT * 4u + 127u) & ~127u);
    bytes = off_js + 2u * NT * 16u + 10u * 8u;
    return (int)bytes <= max_smem;
}

}  // namespace rows
}  // namespace cslbm
