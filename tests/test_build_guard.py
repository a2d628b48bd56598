"""The build refuses force-walk kernels that spill to a local-memory stack frame."""
from paper_0912_1786_gb300 import build

LOG = """ptxas info    : Compiling entry function '_Z6k_walkILb0ELb1EEv' for 'sm_103a'
ptxas info    : Function properties for _Z6k_walkILb0ELb1EEv
    40 bytes stack frame, 36 bytes spill stores, 36 bytes spill loads
ptxas info    : Compiling entry function '_Z6k_walkILb1ELb1EEv' for 'sm_103a'
ptxas info    : Function properties for _Z6k_walkILb1ELb1EEv
    0 bytes stack frame, 0 bytes spill stores, 0 bytes spill loads
ptxas info    : Compiling entry function '_Z7k_otherv' for 'sm_103a'
    16 bytes stack frame, 0 bytes spill stores, 0 bytes spill loads
"""


def test_spilling_walk_variants_are_found():
    bad = build._spilling_kernels(LOG, "k_walk")
    assert bad == [("_Z6k_walkILb0ELb1EEv", 40)]


def test_clean_log_passes():
    assert build._spilling_kernels(LOG.replace("40 bytes stack", "0 bytes stack"), "k_walk") == []
