"""Run PTCA sweeps of a chosen workload, for profilers (ncu) and quick timing.

    python -m paper_1502_07028_gb300.profile_sweep --precision mixed --L 100 --Lc 8 --sweeps 1

Prints one line with the device time of the call and the sweep statistics.
"""
from __future__ import annotations

import argparse
import os
import sys


def parser() -> argparse.ArgumentParser:
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--L", type=int, default=100)
    ap.add_argument("--Lc", type=int, default=8)
    ap.add_argument("--Lz", type=int, default=1, help="third extent (cubic lattice L x L x Lz)")
    ap.add_argument("--Ly", type=int, default=0, help="second extent (0: L; 1: a chain of L sites)")
    ap.add_argument("--offset", type=int, default=-1, help="update-site offset in the window (-1: the default)")
    ap.add_argument("--open", action="store_true", help="open lattice (clipped windows)")
    ap.add_argument("--schedule", choices=["block", "tiled"], default="block")
    ap.add_argument("--stride", type=int, default=0)
    ap.add_argument("--pipeline", choices=["stages", "persistent", "graph", "overlap"], default="graph")
    ap.add_argument("--warps", type=int, choices=[1, 4, 8], default=8, help="warps per CTA of the sweep kernels")
    ap.add_argument("--ctas-per-sm", type=int, default=0, help="persistent CTAs per SM (0: as many as fit)")
    ap.add_argument("--margin", type=float, default=None, help="mixed-mode re-solve margin (0 = off)")
    ap.add_argument("--sweeps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=0)
    ap.add_argument("--T", type=float, default=0.05)
    ap.add_argument("--mu", type=float, default=-6.5)
    ap.add_argument("--JH", type=float, default=8.0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--model", choices=["de", "hubbard", "holstein"], default="de",
                    help="double exchange, the Hubbard mean-field model of Eq. 1, or the Holstein model")
    ap.add_argument("--lam", type=float, default=1.5, help="Holstein electron-lattice coupling")
    ap.add_argument("--K", type=float, default=1.0, help="Holstein elastic constant")
    ap.add_argument("--U", type=float, default=8.0, help="Hubbard U (model hubbard)")
    ap.add_argument("--m-step", type=float, default=0.5, help="field proposal radius (model hubbard)")
    return ap


def config(a):
    """The problem of parsed arguments `a` (30-degree cone proposals)."""
    import paper_1502_07028_gb300 as P
    return P.Config(Lx=a.L, Ly=a.Ly or a.L, Lz=a.Lz, L_c=a.Lc, update_offset=a.offset, periodic=0 if a.open else 1,
                    J_H=a.JH, mu=a.mu, T=a.T, seed=a.seed,
                    schedule=P.SCHEDULE_BLOCK if a.schedule == "block" else P.SCHEDULE_TILED, stride=a.stride,
                    precision=P.MIXED if a.precision == "mixed" else P.FP64, proposal=P.PROPOSAL_CONE,
                    cone_deg=30.0,
                    model={"de": P.MODEL_DOUBLE_EXCHANGE, "hubbard": P.MODEL_HUBBARD_MF,
                           "holstein": P.MODEL_HOLSTEIN}[a.model], U=a.U, m_step=a.m_step, lam=a.lam, K=a.K)


def main(argv=None):
    a = parser().parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import paper_1502_07028_gb300 as P
    from paper_1502_07028_gb300 import _build

    _build.build()
    cfg = config(a)
    ctx = P.Context(cfg)
    P.ptca_set_launch_config(ctx.h, {"stages": P.PIPELINE_STAGES, "persistent": P.PIPELINE_PERSISTENT,
                                     "graph": P.PIPELINE_GRAPH, "overlap": P.PIPELINE_OVERLAP}[a.pipeline], a.warps, a.ctas_per_sm)
    if a.margin is not None and cfg.precision == P.MIXED:
        P.ptca_set_resolve_margin(ctx.h, a.margin)
    if a.warmup:
        ctx.sweep(a.warmup)
    st = ctx.sweep(a.sweeps)
    print(f"{a.precision} {a.model} L={a.L} Lz={a.Lz} Lc={a.Lc} {a.schedule} {a.pipeline} {a.warps} warps: {st.seconds * 1e3:.3f} ms for "
          f"{a.sweeps} sweep(s), "
          f"{cfg.N * a.sweeps / st.seconds:.0f} spin-updates/s, accepted {st.accepted}, resolved {st.resolved}")
    ctx.close()


if __name__ == "__main__":
    main()
