// Host build of the library's integer conversions (csrc/fp_convert.h) for
// the CPU test: reads binary64 values from stdin-sized binary file argv[1],
// writes f64_to_f32_rn of each to argv[2] and f32_to_f64 of those to argv[3].
#include <cstdio>
#include <vector>

#include "fp_convert.h"

int main(int argc, char** argv)
{
    if (argc != 4) return 2;
    FILE* fi = fopen(argv[1], "rb");
    if (!fi) return 3;
    std::vector<double> in;
    double v;
    while (fread(&v, 8, 1, fi) == 1) in.push_back(v);
    fclose(fi);
    std::vector<float> o32(in.size());
    std::vector<double> o64(in.size());
    for (size_t i = 0; i < in.size(); i++) {
        o32[i] = cslbm::f64_to_f32_rn(in[i]);
        o64[i] = cslbm::f32_to_f64(o32[i]);
    }
    FILE* f1 = fopen(argv[2], "wb");
    FILE* f2 = fopen(argv[3], "wb");
    if (!f1 || !f2) return 4;
    fwrite(o32.data(), 4, o32.size(), f1);
    fwrite(o64.data(), 8, o64.size(), f2);
    fclose(f1);
    fclose(f2);
    return 0;
}
