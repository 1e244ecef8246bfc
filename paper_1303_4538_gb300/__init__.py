"""GB300-native Stone SIP solver (hand-written sm_103a CUDA behind a C ABI).

The compute path is the shared library built from ``csrc/`` (see
``paper_1303_4538_gb300.sip``); ``workloads`` draws seeded synthetic systems.
"""
__all__ = ["sip", "workloads"]
