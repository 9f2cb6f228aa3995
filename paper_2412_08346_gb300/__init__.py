"""GB300-native AS-ICP grasp matching ("Grasping by Parallel Shape Matching", arXiv 2412.08346)."""
