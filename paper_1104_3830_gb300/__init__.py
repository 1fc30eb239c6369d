"""GB300-native Sinkhorn preprocessing for the optimal assignment problem
(Sharify, Gaubert, Grigori, arXiv:1104.3830): log-domain Sinkhorn scaling of A^(p)
under an increasing p schedule, threshold pruning, CSR compaction and an exact solve of
the reduced instance with an LP-duality certificate, behind the C ABI of
include/sa.h (libsa.so, sm_103a)."""
from .api import (Context, matrix, sa_assign, sa_assign_host, sa_certify, sa_create, sa_destroy,  # noqa: F401
                  sa_last_error, sa_narrow_i32_to_i16, sa_prune, sa_scale, sa_solve_reduced, sa_verify,
                  sa_version, to_device)
from ._lib import SaError  # noqa: F401
