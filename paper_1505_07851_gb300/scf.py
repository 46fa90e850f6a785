"""SCF-sequence driver for the CG threshold schemes of Section 4b-i.

Host orchestration of the public API only: every step runs in the library
(pcm_esp, pcm_solve, pcm_energy).  Given the densities P_n of an SCF and
the DIIS errors e_n it reports, Eq. 1 is solved at every iteration with the
CG threshold of one of three schemes:

  fixed    delta_tight at every iteration;
  2delta   the "2-delta switching threshold": 1e4 * delta_tight until the
           previous iteration's DIIS error has reached 1e-3, then delta_tight
           (pcm_solve with PCM_TWO_DELTA);
  dynamic  Eq. 21 from the previous DIIS error, evaluated by pcm_solve
           (delta = 1 at the first iteration, when there is none);

optionally starting each solve from the previous iteration's charges.
"""
from __future__ import annotations

SCHEMES = ("fixed", "2delta", "dynamic")


def run_sequence(ctx, seq, scheme, delta_tight=1e-6, warm=True, keep_q=False):
    """Solve Eq. 1 along an SCF history on a Context whose surface and basis
    are set.  seq: [(P_n, e_n), ...] (NumPy arrays or CUDA tensors).
    Returns one record per iteration: the threshold used, the CG steps,
    convergence, the energy of Eq. 13 and (with timing) the solve time;
    with keep_q also a copy of the charges ("q", library point order)."""
    if scheme not in SCHEMES:
        raise ValueError("scheme must be one of %s" % (SCHEMES,))
    out = []
    prev = -1.0
    q = None
    for n, (P, e) in enumerate(seq):
        ctx.esp(P)
        if scheme == "fixed":
            delta, pe = delta_tight, -1.0
        elif scheme == "2delta":
            delta, pe = delta_tight, prev
        else:
            delta, pe = -1.0, prev
        start = warm and q is not None
        q, st = ctx.solve(delta=delta, prev_diis_error=pe, q=q if start else None, warm=start, like=P,
                          two_delta=(scheme == "2delta"))
        E = ctx.energy(q)
        out.append({"iteration": n, "diis_error": e, "delta": st["delta"], "cg_steps": st["iterations"],
                    "converged": bool(st["converged"]), "energy": E, "solve_ms": st["ms_solve"],
                    "refinements": st["refinements"]})
        if keep_q:
            out[-1]["q"] = q.clone() if hasattr(q, "clone") else q.copy()
        prev = e
    return out
