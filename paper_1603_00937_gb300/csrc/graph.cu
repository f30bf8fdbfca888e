// Hamiltonian, graph and partition entry points (device kernels follow in this file).
#include "gbe_internal.h"

extern "C" int gbe_build_hamiltonian(gbe_ctx*, const gbe_sites*, const gbe_tb_model*, gbe_hamiltonian**) {
    gbe_set_error("gbe_build_hamiltonian: not built yet");
    return GBE_EINVAL;
}
extern "C" int gbe_hamiltonian_csr(const gbe_hamiltonian*, gbe_csr*) { return GBE_EINVAL; }
extern "C" int gbe_free_hamiltonian(gbe_hamiltonian*) { return GBE_OK; }
extern "C" int gbe_build_graph(gbe_ctx*, const gbe_csr*, const gbe_graph_params*, gbe_graph**) {
    gbe_set_error("gbe_build_graph: not built yet");
    return GBE_EINVAL;
}
extern "C" int gbe_graph_size(gbe_ctx*, gbe_graph*, int64_t*, int64_t*) { return GBE_EINVAL; }
extern "C" int gbe_graph_export(gbe_ctx*, gbe_graph*, int64_t*, int32_t*) { return GBE_EINVAL; }
extern "C" int gbe_free_graph(gbe_graph*) { return GBE_OK; }
extern "C" int gbe_partition(gbe_ctx*, const gbe_graph*, const gbe_partition_params*, gbe_parts**) {
    gbe_set_error("gbe_partition: not built yet");
    return GBE_EINVAL;
}
