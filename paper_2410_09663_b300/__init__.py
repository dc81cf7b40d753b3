"""paper_2410_09663_b300 -- B300-native Kalman-MPC (placeholder, binding added next)."""
