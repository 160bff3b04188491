"""FP64 CPU oracle of the FPS-SFT recovery loop (test infrastructure only; see fpssft_oracle)."""
