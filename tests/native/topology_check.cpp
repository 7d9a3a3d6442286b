// Runs the library's host-side topology of a general tetrahedral mesh (the part
// of lbm_mesh_upload that needs no GPU) on a mesh read from a binary file and
// writes what it built, for comparison with the CPU oracle.
//   input : int32 N, int32 T, double xyz[N*3], int32 tets[T*4]
//   output: one line "error <message>" or, in binary, int32 counts
//           (nrowptr, ncol, ntris, nbidx) then rowptr, col, tris, bidx and double L
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "lbm_host.h"

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* in = fopen(argv[1], "rb");
    if (!in) return 3;
    int32_t N = 0, T = 0;
    if (fread(&N, 4, 1, in) != 1 || fread(&T, 4, 1, in) != 1) return 4;
    std::vector<double> xyz(3 * (size_t)N);
    std::vector<int32_t> tets(4 * (size_t)T);
    if (fread(xyz.data(), 8, xyz.size(), in) != xyz.size()) return 5;
    if (fread(tets.data(), 4, tets.size(), in) != tets.size()) return 6;
    fclose(in);
    lbm::GeneralTopology g;
    const std::string why = lbm::host_general_topology(N, T, tets.data(), xyz.data(), g);
    FILE* out = fopen(argv[2], "wb");
    if (!out) return 7;
    if (!why.empty()) {
        fprintf(out, "error %s\n", why.c_str());
        fclose(out);
        return 0;
    }
    const int32_t counts[4] = {(int32_t)g.rowptr.size(), (int32_t)g.col.size(), (int32_t)g.tris.size(),
                               (int32_t)g.bidx.size()};
    fwrite("ok", 1, 2, out);
    fwrite(counts, 4, 4, out);
    fwrite(g.rowptr.data(), 4, g.rowptr.size(), out);
    fwrite(g.col.data(), 4, g.col.size(), out);
    fwrite(g.tris.data(), 4, g.tris.size(), out);
    fwrite(g.bidx.data(), 4, g.bidx.size(), out);
    fwrite(&g.L, 8, 1, out);
    fclose(out);
    return 0;
}
