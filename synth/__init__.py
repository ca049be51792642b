"""Seeded synthetic workloads for the POD-2G-PCG solver: structured-mesh FE systems,
KL coefficient fields, loads, snapshot sets and POD bases. Shared input generator for
the oracle and the CUDA path; it holds none of the solver's (PCG / two-grid) arithmetic."""
