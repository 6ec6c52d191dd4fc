"""CPU oracle (test infrastructure only; see ans_oracle)."""
from .ans_oracle import (DCSR, QUANTITY_NAMES, batch, empty_dcsr, link_keys, network_quantities,
                         quantities_array, sum_matrices, traffic_matrix, window_quantities)

__all__ = ["DCSR", "QUANTITY_NAMES", "batch", "empty_dcsr", "link_keys", "network_quantities",
           "quantities_array", "sum_matrices", "traffic_matrix", "window_quantities"]
