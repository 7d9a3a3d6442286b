// Runs the library's host set-up of the space-transformation open boundary and
// writes what it built, for comparison with the CPU oracle.
//   input : int32 n, a, s; double cell
//   output: "error <message>\n", or "ok" then int32 N, nnz, n_outer, n_magnet, shell_tets,
//           rowptr[N+1], col[nnz], outer, magnet, then double K[nnz]
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "lbm_host.h"

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* in = fopen(argv[1], "rb");
    if (!in) return 3;
    int32_t p[3];
    double cell = 0.0;
    if (fread(p, 4, 3, in) != 3 || fread(&cell, 8, 1, in) != 1) return 4;
    fclose(in);
    lbm::ShellGrid G;
    const std::string why = lbm::host_shell_setup(p[0], p[1], p[2], cell, G);
    FILE* out = fopen(argv[2], "wb");
    if (!out) return 5;
    if (!why.empty()) {
        fprintf(out, "error %s\n", why.c_str());
        fclose(out);
        return 0;
    }
    fwrite("ok", 1, 2, out);
    const int32_t h[5] = {(int32_t)G.rowptr.size() - 1, (int32_t)G.col.size(), (int32_t)G.outer.size(),
                          (int32_t)G.magnet.size(), (int32_t)G.shell_tets};
    fwrite(h, 4, 5, out);
    fwrite(G.rowptr.data(), 4, G.rowptr.size(), out);
    fwrite(G.col.data(), 4, G.col.size(), out);
    fwrite(G.outer.data(), 4, G.outer.size(), out);
    fwrite(G.magnet.data(), 4, G.magnet.size(), out);
    fwrite(G.K.data(), 8, G.K.size(), out);
    fclose(out);
    return 0;
}
