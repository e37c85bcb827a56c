"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark."""
from .grids import Case, make_case, tiny, rt617, mid, batch, dayahead, load_profiles, random_point, \
    proportional_dispatch, find_bridges, lp_start, with_loads, horizon_slice, with_transformers, \
    with_block_bids, with_commitment  # noqa: F401
