"""Exact co-mining of delta-temporal motifs on B300 (sm_103a).

The CUDA library is loaded lazily by :mod:`paper_2507_14813_b300.tmotif`;
importing this package loads nothing.
"""
