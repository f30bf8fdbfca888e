/* The C ABI driven from plain C (test program): sites -> H -> graph -> partition -> SP2
 * -> D, every step in libgbe's CUDA kernels, host buffers in and out.
 *
 *   sp2_lattice <in.bin> <out.bin> <h2_thresh> <ncell> <prec>
 *
 * in.bin:  int64 n, double box[3], double pos[n][3], double onsite[n]
 * out.bin: int32 iters, int32 stop, double eps_min, eps_max, int64 n, int64 width,
 *          int32 col[n][width], double val[n][width]   (row i of the ELL = column i of D)
 * Graph |H^2| >= h2_thresh (Eq. 2), cores from ncell^3 spatial cells, SP2 with global
 * traces to the stall stop (Sec. II.A), D assembled column by column (Eq. 6). */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "gbe.h"

#define TRY(call)                                                                          \
    do {                                                                                   \
        int rc_ = (call);                                                                  \
        if (rc_ != GBE_OK) {                                                               \
            fprintf(stderr, "%s failed: %s (%s)\n", #call, gbe_strerror(rc_), gbe_last_error_message()); \
            return 2;                                                                      \
        }                                                                                  \
    } while (0)

static int read_all(FILE* f, void* p, size_t bytes) { return fread(p, 1, bytes, f) == bytes ? 0 : -1; }

int main(int argc, char** argv) {
    if (argc != 6) {
        fprintf(stderr, "usage: %s in.bin out.bin h2_thresh ncell prec\n", argv[0]);
        return 1;
    }
    FILE* fi = fopen(argv[1], "rb");
    if (!fi) return 1;
    int64_t n = 0;
    double box[3];
    if (read_all(fi, &n, 8) || n <= 0 || read_all(fi, box, sizeof(box))) return 1;
    double* pos = (double*)malloc((size_t)n * 3 * sizeof(double));
    double* onsite = (double*)malloc((size_t)n * sizeof(double));
    if (!pos || !onsite || read_all(fi, pos, (size_t)n * 3 * 8) || read_all(fi, onsite, (size_t)n * 8)) return 1;
    fclose(fi);
    const double thresh = atof(argv[3]);
    const int ncell = atoi(argv[4]), prec = atoi(argv[5]);

    gbe_ctx* ctx = NULL;
    TRY(gbe_create(&ctx, 0, NULL));
    gbe_sites st = {n, pos, onsite, {box[0], box[1], box[2]}, 0};
    gbe_tb_model model = {1.0, 2.5, 0.3, -1.0};
    gbe_hamiltonian* Hh = NULL;
    TRY(gbe_build_hamiltonian(ctx, &st, &model, &Hh));
    gbe_csr H;
    TRY(gbe_hamiltonian_csr(Hh, &H));
    gbe_graph_params gp = {GBE_GRAPH_H2_THRESH, thresh, 1, NULL, NULL, NULL, 0.0, 0.0};
    gbe_graph* S = NULL;
    TRY(gbe_build_graph(ctx, &H, &gp, &S));
    gbe_partition_params pp = {GBE_PART_SPATIAL_CELLS, {ncell, ncell, ncell}, &st, 0, 0};
    gbe_parts* parts = NULL;
    TRY(gbe_partition(ctx, S, &pp, &parts));
    gbe_sp2_params prm = {0};
    prm.n_occ = 0.5 * (double)n;
    prm.idem_tol = 1e-10;
    prm.n_min = 10;
    prm.n_max = 100;
    prm.prec = prec;
    prm.branch_mode = GBE_BRANCH_GLOBAL_TRACE;
    gbe_subs* X = NULL;
    gbe_sp2_report rep;
    TRY(gbe_sp2_submatrices(ctx, &H, parts, &prm, &X, &rep));
    gbe_ell D = {n, 0, NULL, NULL, 0};
    TRY(gbe_assemble_D(ctx, X, parts, 0.0, &D));   /* width query */
    D.col = (int32_t*)malloc((size_t)n * D.width * sizeof(int32_t));
    D.val = (double*)malloc((size_t)n * D.width * sizeof(double));
    if (!D.col || !D.val) return 1;
    TRY(gbe_assemble_D(ctx, X, parts, 0.0, &D));   /* host buffers: staged through the device */

    FILE* fo = fopen(argv[2], "wb");
    if (!fo) return 1;
    const int32_t head[2] = {rep.iters, rep.stop_reason};
    fwrite(head, 4, 2, fo);
    fwrite(&rep.eps_min, 8, 1, fo);
    fwrite(&rep.eps_max, 8, 1, fo);
    fwrite(&D.n, 8, 1, fo);
    fwrite(&D.width, 8, 1, fo);
    fwrite(D.col, 4, (size_t)(n * D.width), fo);
    fwrite(D.val, 8, (size_t)(n * D.width), fo);
    fclose(fo);
    printf("iters %d stop %d width %lld\n", rep.iters, rep.stop_reason, (long long)D.width);

    free(D.col);
    free(D.val);
    TRY(gbe_free_subs(X));
    TRY(gbe_free_parts(parts));
    TRY(gbe_free_graph(S));
    TRY(gbe_free_hamiltonian(Hh));
    TRY(gbe_destroy(ctx));
    free(pos);
    free(onsite);
    return 0;
}
