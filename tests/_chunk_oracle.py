"""Worker of the full-size parity test: one chunk of the counter-based shower
evaluated by the oracle at a few antennas.  A module of its own (numpy, the
oracle and the generator twin only) so that spawned worker processes import it
without the GPU stack."""
import numpy as np

import oracle
from paper_2309_03717_gb300 import synth


def chunk_job(job):
    """job = (first, n, seed, zenith_deg, ant_xyz, t_start_ns, n_bins, dt_ns, medium, formalism).
    Returns (global indices of the tracks left out, traces [n_sample, 3, n_bins]
    summed over the chunk, kept count).  Left out: tracks with an arrival within
    1e-6 bin of an edge at a sampled antenna (either bin is correct there); they
    get charge 0 on both sides, so the track filter drops them."""
    first, n, seed, zenith, ant, t_start_ns, n_bins, dt_ns, medium, formalism = job
    tr = oracle.tracks_from_ns(synth.make_tracks_counter(first, n, seed, zenith))
    form = oracle.ENDPOINT if formalism == "endpoint" else oracle.ZHS
    t_ref = np.asarray(t_start_ns) * 1e-9
    _, u = oracle.arrivals(tr, ant, t_ref, n_bins, dt_ns * 1e-9, medium, form)
    fr = u - np.floor(u)
    amb = (np.minimum(fr, 1.0 - fr) < 1e-6).reshape(n, -1).any(axis=1)
    tr["q"] = np.where(amb, 0.0, tr["q"])
    out, kept = oracle.forward(tr, ant, t_ref, n_bins, dt_ns * 1e-9, medium, form)
    return first + np.nonzero(amb)[0], out, kept
