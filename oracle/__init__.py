"""FP64 CPU oracle for the QuasiGrad hot path.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the library's product path.
"""
from .qg_oracle import evaluate, objective, unpack, unpack_u, pack, box, device_sign, energy_cost, ac_flows, bus_mismatch, dc_network, \
    dc_injections, dc_base_flows, soft_abs, soft_relu, TERM_NAMES  # noqa: F401
from .adam import adam_step, normalized_time, magnitude_scale, step_size, schedule_table  # noqa: F401
