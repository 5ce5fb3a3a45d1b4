// Host build of the row passes' plan (csrc/rows_plan.h) for the CPU test:
// reads n0 n1 n2 yper zper s_bytes max_smem and prints the plan's fields.
#include <cstdio>
#include <cstdlib>

#include "rows_plan.h"

int main(int argc, char** argv)
{
    if (argc != 8) return 2;
    const int n[3] = {atoi(argv[1]), atoi(argv[2]), atoi(argv[3])};
    const bool yper = atoi(argv[4]) != 0, zper = atoi(argv[5]) != 0;
    const int sb = atoi(argv[6]), max_smem = atoi(argv[7]);
    cslbm::rows::Plan pl{};
    const bool ok = cslbm::rows::make_plan(n, yper, zper, sb, max_smem, pl);
    unsigned off_m = 0, off_sg = 0, off_h4 = 0, off_js = 0, fbytes = 0;
    const bool fok = ok && cslbm::rows::fused_layout(pl, sb, max_smem, off_m, off_sg, off_h4, off_js, fbytes);
    printf("ok=%d TR=%d nyb=%d y1=%d z0=%d ntiles=%d JS=%d JL=%d JR=%d off_jf=%u off_geo=%u off_hist=%u "
           "stage=%u smem=%u fused_ok=%d off_m=%u off_sg=%u off_h4=%u off_js=%u fused=%u\n",
           ok, pl.TR, pl.nyb, pl.y1, pl.z0, pl.ntiles, pl.JS, pl.JL, pl.JR, pl.off_jf, pl.off_geo, pl.off_hist,
           pl.stage_bytes, ok ? cslbm::rows::smem_bytes(pl) : 0u, fok, off_m, off_sg, off_h4, off_js, fbytes);
    return 0;
}
