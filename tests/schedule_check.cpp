// Host-side check of the persistent 3-D step schedule, built from the library's own
// sources: plan_persistent (tmap.cpp) fills a launch's schedule, schedule_segment
// (step3d.h) enumerates what each CTA streams, and every (tile column, output plane) must
// be computed exactly once.  Prints "ok <combinations>" or the first failure.
#include <cstdio>
#include <vector>

#include "step3d.h"

int main()
{
    const int nzs[] = {20, 33, 64, 100, 296, 440, 552, 1000};
    const int Ms[] = {4, 8};
    const int colss[] = {1, 2, 3, 50, 95, 151, 152, 153, 162, 200, 303, 304, 305, 315, 607,
                         608, 609, 1000};
    const int residents[] = {1, 7, 152, 304, 456, 608};
    int combos = 0;
    for (int nz : nzs)
        for (int M : Ms)
            for (int columns : colss)
                for (int resident : residents)
                    for (int in_step = 0; in_step < 2; ++in_step) {
                        fwi::Step3dParams p{};
                        p.M = M;
                        p.nz = nz;
                        const int grid = fwi::plan_persistent(p, columns, resident, in_step != 0);
                        if (grid < 1 || grid > resident) {
                            std::printf("bad grid %d: nz %d M %d columns %d resident %d in_step %d\n",
                                        grid, nz, M, columns, resident, in_step);
                            return 1;
                        }
                        std::vector<unsigned char> seen((size_t)columns * nz, 0);
                        for (int k = 0; k < grid; ++k) {
                            int col, z0, z1;
                            for (int idx = 0; fwi::schedule_segment(p, columns, k, idx, &col, &z0, &z1); ++idx) {
                                if (col < 0 || col >= columns || z0 < 0 || z1 > nz || z0 >= z1) {
                                    std::printf("bad segment (%d, %d, %d): nz %d M %d columns %d resident %d in_step %d\n",
                                                col, z0, z1, nz, M, columns, resident, in_step);
                                    return 1;
                                }
                                for (int z = z0; z < z1; ++z) ++seen[(size_t)col * nz + z];
                            }
                        }
                        for (size_t i = 0; i < seen.size(); ++i)
                            if (seen[i] != 1) {
                                std::printf("column %zu plane %zu computed %d times: nz %d M %d columns %d "
                                            "resident %d in_step %d\n",
                                            i / nz, i % nz, (int)seen[i], nz, M, columns, resident, in_step);
                                return 1;
                            }
                        ++combos;
                    }
    std::printf("ok %d\n", combos);
    return 0;
}
