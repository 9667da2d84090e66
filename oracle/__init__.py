"""FP64 CPU oracle of the TPC sector tracker -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  The product path (paper_1910_12214_b300) never does.
"""
from .oracle import (CODE_FIELDS, MASK_ASSOCIATED, MASK_PROTECTED, MASK_REMOVE_A, MASK_REMOVE_B,  # noqa: F401
                     MLP_NP, OracleConfig, adam, bf16, build_oracle, chi2, cluster_masks, code_stream, compress,
                     correct_clusters, counter_uniform, decode_stream, decompress, dyn_round, encode_clusters,
                     fit_hits, grid_order, join_loopers, mask_thresholds, merge, merge_tracks, mlp_batch, mlp_forward,
                     mlp_grad, mlp_init,
                     oracle_tracks, predict_codes, propagate, run, trilinear)
