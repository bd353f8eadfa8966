"""Host-side arithmetic of bench.py that needs no GPU."""
import bench


def test_binding_roof_follows_the_machine_balance():
    # 80.5 TFLOP/s over 6.78 TB/s: the balance is 11.9 flop/B
    assert bench.binding_roof(81.3, 939, 6777.3, 80.5) == "hbm"      # 11.5 flop/B
    assert bench.binding_roof(81.3, 1142, 6777.3, 80.5) == "alu"     # 14.0 flop/B
    assert bench.binding_roof(1.0, 0.0, 6777.3, 80.5) == "hbm"
    assert bench.binding_roof(0.0, 1.0, 6777.3, 80.5) == "alu"
