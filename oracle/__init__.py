"""FP64 CPU oracle for OCD detection: test infrastructure, never the product path."""
from .ocd import (  # noqa: F401
    BOX,
    MMSE,
    alphabet,
    bits_per_symbol,
    box_qp_bruteforce,
    box_radius,
    cd_equalize,
    exact_mu_rho,
    hard_bits,
    maxlog_mimo_exhaustive,
    mmse_closed_form,
    objective,
    ocd_detect,
    ocd_equalize,
    ocd_llr,
    preprocess,
    project,
)
from .unfolded import bce_loss, maxlog_llr, unfolded_forward, unfolded_loss_and_grad  # noqa: F401,E402
