"""GB300-native (sm_103a) per-vertex orbit counting of all connected 2- to
5-vertex graphlets, after EVOKE (Pashanasangi & Seshadhri).

Public API (CUDA only; no CPU fallback):
    count_orbits(rowptr, colidx, n, m)  -> int64 [n, 73] induced orbit counts
    edge_orbits(rowptr, colidx, n, m)   -> per-edge T, C4, K4, E7, E9
    edge_orbit_counts(rowptr, colidx, n, m) -> per-slot E0..E11 (Lem. 4edgeorbit)
    build_dag(rowptr, colidx, n, m)     -> degree-ordered DAG
    count_batch(rowptr_cat, colidx_cat, vtx_off, edge_off) -> counts of many graphs
    Plan.single / Plan.batch            -> sized plans: execute(), launch_graph()
    orbit_matrix()                      -> the 73x73 matrix A (DM = A DIM)
    graphlet_totals(counts)             -> global pattern counts from orbit counts
"""
from ._lib import (EvokeError, Plan, batch_to_device, build_dag, count_batch, count_orbits,
                   edge_orbit_counts, edge_orbits, graphlet_totals, load, orbit_matrix, to_device, version)

__all__ = ["EvokeError", "Plan", "batch_to_device", "build_dag", "count_batch", "count_orbits",
           "edge_orbit_counts", "edge_orbits", "graphlet_totals", "load", "orbit_matrix", "to_device", "version"]
