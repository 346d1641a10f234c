// Contraction-tree executor (qcs_contract_tree, qcs_contract_tree_backward).
#include "internal.h"

extern "C" {

int qcs_contract_tree(qcs_handle_t h, const qcs_tree_t *tree, const qcs_c32 *const *leaves,
                      double *d_out, qcs_run_info_t *info) {
    (void)h; (void)tree; (void)leaves; (void)d_out; (void)info;
    return QCS_ERR_UNSUPPORTED;
}

int qcs_contract_tree_backward(qcs_handle_t h, const qcs_tree_t *tree,
                               const qcs_c32 *const *leaves, const double *d_grad_out,
                               qcs_c32 *const *d_grad_leaves, qcs_run_info_t *info) {
    (void)h; (void)tree; (void)leaves; (void)d_grad_out; (void)d_grad_leaves; (void)info;
    return QCS_ERR_UNSUPPORTED;
}

}
