// Host build of the coefficient generator's FP64 ray walk (walk.cuh) for the
// CPU test suite.  It traces rays of one view on the CPU with the same walk
// the generator kernel runs and prints each row, so that the tests can compare
// the walk's logic with the oracle's direct trace without a GPU.
//
// Usage: host_walk geometry n_rings n_slabs sector_rule r h z_min n_views
//                  arc_num arc_den n_u n_v du dv d_so d_sd view ray_begin ray_end
// Output, one line per ray: "ray bound n cell_0 w_0 cell_1 w_1 ..." with the
// FP32 sizing pass's bound on the row's length (size_ray), then the walk's
// entries: global cell ids (slab * cells_per_slab + head + sector) and FP64
// lengths (%.17g), in the walk's order.
#include <math.h>  // the walk calls cos, sin, sqrt, floor, atan2 unqualified

#include "../paper_2208_12964_gb300/csrc/walk.cuh"

#include <cstdio>
#include <cstdlib>
#include <vector>

using namespace uspg;

int main(int argc, char **argv)
{
    if (argc != 20) {
        std::fprintf(stderr, "usage: see the header of host_walk.cpp\n");
        return 2;
    }
    Geometry g{};
    g.geometry = std::atoi(argv[1]);
    g.n_rings = std::atoi(argv[2]);
    g.n_slabs = std::atoi(argv[3]);
    int rule = std::atoi(argv[4]);
    g.r = std::atof(argv[5]);
    g.h = std::atof(argv[6]);
    g.z_min = std::atof(argv[7]);
    g.n_views = std::atoi(argv[8]);
    g.arc_num = std::atoll(argv[9]);
    g.arc_den = std::atoll(argv[10]);
    g.n_u = std::atoi(argv[11]);
    g.n_v = std::atoi(argv[12]);
    g.du = std::atof(argv[13]);
    g.dv = std::atof(argv[14]);
    g.d_so = std::atof(argv[15]);
    g.d_sd = std::atof(argv[16]);
    int view = std::atoi(argv[17]), r0 = std::atoi(argv[18]), r1 = std::atoi(argv[19]);
    if (g.geometry != USPG_CONE_3D) g.n_slabs = 1;
    g.n_rays = g.n_u * (g.geometry == USPG_CONE_3D ? g.n_v : 1);
    g.n_rows = g.n_rays;
    g.weight_mode = USPG_LENGTH;
    // ring table and boundary directions, as the library builds them
    const int N = g.n_rings;
    std::vector<RingEntry> rt(N);
    long long head = 0;
    for (int i = 0; i < N; i++) {
        int n = i + 1;
        rt[i].ng = rule == USPG_SECT_6N ? 6 * n : 4 * (2 * n - 1);
        rt[i].head = (int)head;
        rt[i].step = 0;
        rt[i].chunk0 = 0;
        head += rt[i].ng;
    }
    g.cells_per_slab = head;
    std::vector<double2> bdir(head);
    std::vector<float2> bdirf(head);
    for (int i = 0; i < N; i++)
        for (int j = 0; j < rt[i].ng; j++) {
            double a = kTwoPi * (double)j / (double)rt[i].ng;
            double c = cos(a), s = sin(a);
            bdir[rt[i].head + j] = make_double2(c, s);
            bdirf[rt[i].head + j] = make_float2((float)c, (float)s);
        }
    const int cap = 1 << 16;
    std::vector<uint32_t> idx(cap), in_cell(N);
    std::vector<double> w(cap), root(N);
    std::vector<int> in_pos(N);
    int status = 0;
    for (int ray = r0; ray < r1; ray++) {
        FillSink sink;
        sink.idx = idx.data();
        sink.w = w.data();
        sink.cap = cap;
        sink.in_cell = in_cell.data();
        sink.in_pos = in_pos.data();
        sink.root = root.data();
        walk_ray(g, rt.data(), bdir.data(), bdirf.data(), view, ray, sink, &status);
        if (sink.overflow) status |= kStatusCountMismatch;
        std::printf("%d %d %d", ray, size_ray(g, rt.data(), bdirf.data(), view, ray), sink.n);
        for (int q = 0; q < sink.n; q++) {
            uint32_t pc = idx[q];
            long long cell = (long long)cell_slab(pc) * g.cells_per_slab + rt[cell_ring(pc)].head + cell_sector(pc);
            std::printf(" %lld %.17g", cell, w[q]);
        }
        std::printf("\n");
    }
    return status ? 3 : 0;
}
