"""Workload definitions: BB codes, noise, decoder presets and seeds.

Plain data only (no decoder arithmetic), so that both the CUDA path and the
CPU oracle used by the tests draw their inputs from the same definitions.

Codes (appendix "Single shot syndrome noise" gives the [[288,12,18]]
polynomials; the others are the bivariate-bicycle family decoded in Fig. 3):
A and B are lists of three monomials x^a y^b as (a, b), in the order the
polynomial is written; that order fixes which term each CNOT layer uses.
"""

CODES = {
    "72": dict(name="[[72,12,6]]", n=72, k=12, d=6, l=6, m=6,
               A=[(3, 0), (0, 1), (0, 2)], B=[(0, 3), (1, 0), (2, 0)]),
    "90": dict(name="[[90,8,10]]", n=90, k=8, d=10, l=15, m=3,
               A=[(9, 0), (0, 1), (0, 2)], B=[(0, 0), (2, 0), (7, 0)]),
    "108": dict(name="[[108,8,10]]", n=108, k=8, d=10, l=9, m=6,
                A=[(3, 0), (0, 1), (0, 2)], B=[(0, 3), (1, 0), (2, 0)]),
    "144": dict(name="[[144,12,12]]", n=144, k=12, d=12, l=12, m=6,
                A=[(3, 0), (0, 1), (0, 2)], B=[(0, 3), (1, 0), (2, 0)]),
    "288": dict(name="[[288,12,18]]", n=288, k=12, d=18, l=12, m=12,
                A=[(3, 0), (0, 2), (0, 7)], B=[(0, 3), (1, 0), (2, 0)]),
}

# Decoder parameters shared by both presets: Alg. 3 thresholds (P_A..P_D),
# the message clip of 50, peeling and shortening to 2w' columns; a window in
# which no decision path converges outputs the estimate with the fewest
# unsatisfied committed checks (fallback 2; Alg. 2 leaves this case open).
_COMMON = dict(W=3, F=1, low_error_mode=0, peel_at_init=1, shorten=1, clip=50.0,
               pa_main=-3.0, pa_other=0.0, pb_main=-12.0, pb_other=-10.0, pb_d1=-16.0,
               pc=30.0, pd=3.0, pc_max_depth=4, n_unsat_min=3, side_max=0, reinit_on_split=0,
               iters_first=0, merge_h1=0, reuse_msgs=0, fallback=2)

# "configured": normalised min-sum alpha = 0.625, 100 BP iterations on the
# full window, decimation steps of 10 iterations, 2^k guessing tree.
CONFIGURED = dict(_COMMON, alpha=0.625, n_pre=100, iters_per_step=10, d_max_main=25)

# "paper": the values of Sec. IV-C and Fig. 2 for N <= 144 (alpha = 1.0, 8
# pre-BP iterations, 6 iterations per step, D_max 25 on the main path, side
# branches splitting off at D_split = k .. 10, every non-main path running 10
# steps past its last guess).
PAPER = dict(_COMMON, alpha=1.0, n_pre=8, iters_per_step=6, d_max_main=25, side_max=10)


# Code-capacity workloads of the appendices (data-qubit noise BSC(p_d) decoded
# with H_X; single-shot syndrome noise with [H_X | I]): one window over the
# whole matrix, no pre-BP and no shortening, alpha = 0.625, low-error mode,
# main branch D_max 40, guessing tree of depth 5, side branches up to
# D_split = 20, every non-main path running 30 steps past its last guess.
CAPACITY = dict(_COMMON, W=1, F=1, alpha=0.625, n_pre=0, iters_per_step=6, d_max_main=40,
                low_error_mode=1, shorten=0, side_max=20, k_guess=5, d_max_other=35)


def preset(name, k_guess, p=None, **over):
    """Decoder parameters; the non-main paths run 10 steps past depth k.
    The "paper" preset of [[288,12,18]] (Sec. IV-C) is
    preset("paper", 5, p, d_max_main=40, d_max_other=25, side_max=20, n_pre=16)."""
    base = {"configured": CONFIGURED, "paper": PAPER}[name]
    out = dict(base, k_guess=k_guess, d_max_other=k_guess + 10)
    if p is not None and p <= 0.002:
        out["low_error_mode"] = 1  # Fig. 3 caption: no Alg. 3 for p <= 0.002
    out.update(over)
    return out


# Seeded synthetic workloads (Monte-Carlo memory experiments).
WORKLOADS = {
    "bb72_r6_p3e-3": dict(code="72", rounds=6, p=0.003, k_guess=3, shots=2000, seed=72_003),
    "bb144_r12_p3e-3": dict(code="144", rounds=12, p=0.003, k_guess=4, shots=100_000,
                            seed=144_003),
}
# [[144,12,12]], 12 rounds, (3,1) windows, k = 4: the physical error rates of
# the LER sweep, 1e5 shots each, seeds 144_00{1..4}
SWEEP_144 = [dict(p=p, seed=144_000 + i, shots=100_000) for i, p in enumerate((0.001, 0.002, 0.003, 0.004), 1)]
