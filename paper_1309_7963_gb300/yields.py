"""Positron-emitter yields from the residual-nucleus tally (pnuc_tally), the application the
paper proposes for range verification (§4.2): for each incident-energy bin, the fraction of
non-elastic events that leave each beta+ emitter as the final residual nucleus."""
from __future__ import annotations

import numpy as np

# beta+ emitters produced on tissue nuclei (C, N, O, P, Ca): (Z, A) -> (name, half-life in s)
POSITRON_EMITTERS = {
    (6, 10): ("10C", 19.3), (6, 11): ("11C", 1221.8), (7, 12): ("12N", 0.011), (7, 13): ("13N", 597.9),
    (8, 14): ("14O", 70.6), (8, 15): ("15O", 122.2), (9, 17): ("17F", 64.5), (9, 18): ("18F", 6586.2),
    (15, 29): ("29P", 4.1), (15, 30): ("30P", 149.9), (19, 37): ("37K", 1.23), (19, 38): ("38K", 458.2),
    (20, 39): ("39Ca", 0.86),
}


def emitter_yields(residual_hist, E_range, min_events: int = 1) -> dict:
    """residual_hist: the [n_E][Z_max + 1][A_max + 1] counts of pnuc_tally (numpy or torch).
    Returns {name: array over energy bins of yield per non-elastic event} and the bin edges;
    bins with fewer than min_events events give NaN."""
    h = residual_hist.cpu().numpy() if hasattr(residual_hist, "cpu") else np.asarray(residual_hist)
    n_E = h.shape[0]
    events = h.reshape(n_E, -1).sum(axis=1).astype(np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        out = {}
        for (Z, A), (name, _) in POSITRON_EMITTERS.items():
            if Z < h.shape[1] and A < h.shape[2]:
                out[name] = np.where(events >= min_events, h[:, Z, A] / events, np.nan)
    return {"edges": np.linspace(E_range[0], E_range[1], n_E + 1), "events": events, "yields": out}
