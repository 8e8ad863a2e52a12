"""The oracle's self-test in plain C (oracle/test_oracle.c): raw sizes of the
paper's spaces, the adjacent example of Sec. III-B, chain and tournament
closed forms, a C_p hand example and the published SplitMix64 outputs."""
import oracle


def test_oracle_c_self_test():
    status, out = oracle.run_self_test()
    assert status == 0, out
    assert "oracle self-checks passed" in out
